"""GB300 (sm_103a) rigid multi-site molecular dynamics hot path (arXiv 1408.4599).

The compute path is the CUDA library ``libmdgpu.so`` behind the C ABI of
``include/md.h``; :mod:`paper_1408_4599_gb300.md` is its thin ctypes binding.
"""
from . import md  # noqa: F401
from .md import (System, md_compute_forces, md_create, md_destroy, md_energy_virial,  # noqa: F401
                 md_get_forces, md_get_molecules, md_kernel_times_get, md_profile, md_set_molecules, md_step,
                 md_sync)
