// md_force_inst.cu -- explicit instantiation of the force kernel launch
// (md_force.cuh) for one compiled signature and one stencil radius.
// build.py compiles this file once per (MD_FORCE_SIG, MD_FORCE_M) pair, so
// that the twelve kernel pairs compile in parallel:
//   MD_FORCE_SIG: 0 1CLJ, 1 2CLJ, 2 2CLJQ, 3 2CLJDQ, 4 4-site, 5 run-time
//   signature (the order of dispatch_sig in md_pair.cuh);
//   MD_FORCE_M: 1 (cells of edge >= r_c) or 2 (>= r_c / 2).
#include <tuple>

#include "md_force.cuh"

#if !defined(MD_FORCE_SIG) || !defined(MD_FORCE_M)
#error "md_force_inst.cu is compiled with -DMD_FORCE_SIG=0..5 -DMD_FORCE_M=1|2 (see build.py)"
#endif

namespace mdk {

using ForceInstSig =
    std::tuple_element_t<MD_FORCE_SIG, std::tuple<Sig1CLJ, Sig2CLJ, Sig2CLJQ, Sig2CLJDQ, Sig4Site, SigDyn>>;
template cudaError_t launch_force_sig<ForceInstSig, MD_FORCE_M>(const ForceArgs &, int, int, cudaStream_t);

}  // namespace mdk
