// md_api.cu -- host side of the C ABI declared in include/md.h: argument
// validation, compilation of the molecular model into the kernels' site
// table, device buffers, launch sequencing of one MD step (§3: cell rebuild
// -> force and torque calculation -> summation -> leapfrog), observables.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/md.h"
#include "md_internal.cuh"

struct PendingTiming {
    int kind;
    cudaEvent_t a, b;
};

// Editable copy of the caller's model (parameters can be replaced later).
struct HostModel {
    int T = 0;
    std::vector<double> eps, sigma, xi, eta;
    int n_lj = 0, n_chg = 0, n_dip = 0, n_quad = 0;
    std::vector<double> lj_pos, lj_mass, chg_pos, chg_q, dip_pos, dip_axis, dip_mu, quad_pos, quad_axis, quad_Q;
    std::vector<int32_t> lj_type;
    bool has_xi = false, has_eta = false;
    md_component comp;
    md_site_types types;
    void view()
    {
        comp = md_component{n_lj, lj_pos.data(), lj_type.data(), lj_mass.data(), n_chg, chg_pos.data(), chg_q.data(),
                            n_dip, dip_pos.data(), dip_axis.data(), dip_mu.data(), n_quad, quad_pos.data(),
                            quad_axis.data(), quad_Q.data()};
        types = md_site_types{T, eps.data(), sigma.data(), has_xi ? xi.data() : nullptr,
                              has_eta ? eta.data() : nullptr, 1, &comp};
    }
};

struct md_system {
    Grid g;
    DevModel m;
    DevState d;
    md_options opt;
    int half_eff;                // half shell actually used (needs >= 3 cells per axis)
    bool acc_zeroed = false;     // the last rebuild cleared the FP32 accumulator records
    int n_force_blocks, n_kin_blocks;
    long long cap;               // allocated molecules
    bool has_mol, binned, forces_valid;
    bool f_in_acc;               // the latest forces exist only in the FP32 accumulators (half shell)
    double dt_last, time;
    long long step;
    cudaStream_t last_stream;
    // host-side model facts for the scalar terms
    double lrc_u_coef, lrc_w_coef;  // U_LRC = coef N^2 / V (the same for W)
    double rf_self_per_mol;
    int n_lj, n_el;
    HostModel hm;
    double rc;
    // electrostatic entities in the adjoint kernel's order (site, then charge/dipole/quadrupole):
    // parameter index and strength; LJ sites in site order: type
    std::vector<int> ent_param, lj_site_type;
    std::vector<double> ent_strength;
    double *adj_partials = nullptr;
    int adj_nacc = 0;
    char err[512];
    // profiling
    bool profiling;
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> pool;
    md_kernel_times times;
    // md_step replays two captured steps per graph launch: one executable
    // graph per buffer parity (the ping-pong state buffers swap every step)
    cudaGraphExec_t gexec[2];
    double gdt[2], gT[2];
    int parity;
};

namespace {

void set_err(md_system *s, const char *fmt, ...)
{
    if (!s) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->err, sizeof s->err, fmt, ap);
    va_end(ap);
}

md_status cuda_fail(md_system *s, cudaError_t e, const char *where)
{
    set_err(s, "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA;
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, where); \
    } while (0)

bool finite3(const double *p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

cudaEvent_t get_event(md_system *s)
{
    if (!s->pool.empty()) {
        cudaEvent_t e = s->pool.back();
        s->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

struct TimeScope {
    md_system *s;
    cudaStream_t st;
    int kind;
    cudaEvent_t a = nullptr;
    TimeScope(md_system *s_, cudaStream_t st_, int kind_) : s(s_), st(st_), kind(kind_)
    {
        if (s->profiling) {
            a = get_event(s);
            if (a) cudaEventRecord(a, st);
        }
    }
    ~TimeScope()
    {
        if (s->profiling && a) {
            cudaEvent_t b = get_event(s);
            if (b) {
                cudaEventRecord(b, st);
                s->pending.push_back({kind, a, b});
            }
        }
    }
};

void drain_timings(md_system *s)
{
    for (auto &p : s->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            s->times.ms[p.kind] += ms;
            s->times.launches[p.kind] += 1;
        }
        s->pool.push_back(p.a);
        s->pool.push_back(p.b);
    }
    s->pending.clear();
}

// ---------------------------------------------------------- model set-up
// Entities of the component are merged into GPU sites: an entity joins an
// existing site at the same position when that site does not yet carry
// its role (and, for dipoles/quadrupoles, has no axis or the same axis).
md_status compile_model(md_system *s, const md_site_types *t, double rc, int lj_shift, double eps_rf)
{
    DevModel &m = s->m;
    memset(&m, 0, sizeof m);
    if (!t || t->n_comp != 1 || !t->comp) {
        set_err(s, "md_site_types: exactly one component is supported (got %d)", t ? t->n_comp : -1);
        return (t && t->n_comp > 1) ? MD_ERR_UNSUPPORTED : MD_ERR_ARG;
    }
    const int T = t->n_types;
    if (T < 0 || T > MD_MAX_TYPES || (T > 0 && (!t->eps || !t->sigma))) {
        set_err(s, "bad LJ type table (n_types=%d)", T);
        return T > MD_MAX_TYPES ? MD_ERR_UNSUPPORTED : MD_ERR_ARG;
    }
    for (int a = 0; a < T; a++) {
        if (!(std::isfinite(t->eps[a]) && t->eps[a] >= 0.0 && std::isfinite(t->sigma[a]) && t->sigma[a] > 0.0)) {
            set_err(s, "LJ type %d: eps must be >= 0 and sigma > 0", a);
            return MD_ERR_ARG;
        }
        for (int b = 0; b < T; b++) {
            double xi = t->xi ? t->xi[a * T + b] : 1.0, eta = t->eta ? t->eta[a * T + b] : 1.0;
            if (!(std::isfinite(xi) && xi >= 0.0 && std::isfinite(eta) && eta > 0.0)) {
                set_err(s, "binary parameters xi/eta must be finite, xi >= 0, eta > 0");
                return MD_ERR_ARG;
            }
        }
    }
    const md_component &c = t->comp[0];
    if (c.n_lj < 0 || c.n_chg < 0 || c.n_dip < 0 || c.n_quad < 0 || (c.n_lj && (!c.lj_pos || !c.lj_type || !c.lj_mass)) ||
        (c.n_chg && (!c.chg_pos || !c.chg_q)) || (c.n_dip && (!c.dip_pos || !c.dip_axis || !c.dip_mu)) ||
        (c.n_quad && (!c.quad_pos || !c.quad_axis || !c.quad_Q))) {
        set_err(s, "md_component: negative count or NULL array");
        return MD_ERR_ARG;
    }
    struct HSite {
        double pos[3];
        int roles;
        int lj_type;
        double q, mu, Q;
        double axis[3];
        bool has_axis;
    };
    std::vector<HSite> sites;
    auto same = [](const double *a, const double *b) {
        return std::fabs(a[0] - b[0]) < 1e-12 && std::fabs(a[1] - b[1]) < 1e-12 && std::fabs(a[2] - b[2]) < 1e-12;
    };
    std::vector<std::vector<int>> site_param(MD_MAX_SITES + 8, std::vector<int>(3, -1));
    int cur_param = -1;
    auto role_idx = [](int role) { return role == ROLE_CHG ? 0 : (role == ROLE_DIP ? 1 : 2); };
    auto add = [&](const double *pos, int role, int ljt, double val, const double *axis) -> md_status {
        if (!finite3(pos) || !std::isfinite(val) || (axis && !finite3(axis))) return MD_ERR_ARG;
        double ax[3] = {0, 0, 0};
        if (axis) {
            double n = std::sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
            if (!(n > 0.0)) return MD_ERR_ARG;
            for (int k = 0; k < 3; k++) ax[k] = axis[k] / n;
        }
        for (auto &h : sites) {
            if (!same(h.pos, pos) || (h.roles & role)) continue;
            if (axis && h.has_axis && !same(h.axis, ax)) continue;
            h.roles |= role;
            if (role == ROLE_LJ) h.lj_type = ljt;
            if (role == ROLE_CHG) h.q = val;
            if (role == ROLE_DIP) h.mu = val;
            if (role == ROLE_QUAD) h.Q = val;
            if (axis && !h.has_axis) {
                memcpy(h.axis, ax, sizeof ax);
                h.has_axis = true;
            }
            size_t si = (size_t)(&h - sites.data());
            if (role != ROLE_LJ && si < site_param.size()) site_param[si][role_idx(role)] = cur_param;
            return MD_OK;
        }
        HSite h;
        memset(&h, 0, sizeof h);
        memcpy(h.pos, pos, sizeof h.pos);
        h.roles = role;
        h.lj_type = ljt;
        if (role == ROLE_CHG) h.q = val;
        if (role == ROLE_DIP) h.mu = val;
        if (role == ROLE_QUAD) h.Q = val;
        if (axis) {
            memcpy(h.axis, ax, sizeof ax);
            h.has_axis = true;
        }
        sites.push_back(h);
        size_t si = sites.size() - 1;
        if (role != ROLE_LJ && si < site_param.size()) site_param[si][role_idx(role)] = cur_param;
        return MD_OK;
    };
    double mass = 0.0, com[3] = {0, 0, 0}, In[9] = {0};
    for (int a = 0; a < c.n_lj; a++) {
        int ty = c.lj_type[a];
        double mm = c.lj_mass[a];
        if (ty < 0 || ty >= T || !(std::isfinite(mm) && mm >= 0.0)) {
            set_err(s, "LJ site %d: type out of range or bad mass", a);
            return MD_ERR_ARG;
        }
        if (add(&c.lj_pos[3 * a], ROLE_LJ, ty, 0.0, nullptr) != MD_OK) {
            set_err(s, "LJ site %d: non-finite position", a);
            return MD_ERR_ARG;
        }
        const double *p = &c.lj_pos[3 * a];
        mass += mm;
        double p2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
        for (int k = 0; k < 3; k++) com[k] += mm * p[k];
        for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++) In[3 * r + q] += mm * ((r == q ? p2 : 0.0) - p[r] * p[q]);
    }
    for (int a = 0; a < c.n_chg; a++)
        if ((cur_param = 2 * T + a, add(&c.chg_pos[3 * a], ROLE_CHG, -1, c.chg_q[a], nullptr)) != MD_OK) {
            set_err(s, "charge %d: non-finite input", a);
            return MD_ERR_ARG;
        }
    for (int a = 0; a < c.n_dip; a++)
        if ((cur_param = 2 * T + c.n_chg + a, add(&c.dip_pos[3 * a], ROLE_DIP, -1, c.dip_mu[a], &c.dip_axis[3 * a])) !=
            MD_OK) {
            set_err(s, "dipole %d: non-finite input or zero axis", a);
            return MD_ERR_ARG;
        }
    for (int a = 0; a < c.n_quad; a++)
        if ((cur_param = 2 * T + c.n_chg + c.n_dip + a,
             add(&c.quad_pos[3 * a], ROLE_QUAD, -1, c.quad_Q[a], &c.quad_axis[3 * a])) != MD_OK) {
            set_err(s, "quadrupole %d: non-finite input or zero axis", a);
            return MD_ERR_ARG;
        }
    if (sites.empty()) {
        set_err(s, "component has no interaction sites");
        return MD_ERR_ARG;
    }
    if ((int)sites.size() > MD_MAX_SITES) {
        set_err(s, "%d merged sites exceed the supported %d", (int)sites.size(), MD_MAX_SITES);
        return MD_ERR_UNSUPPORTED;
    }
    // principal-axes frame and centre of mass at the origin
    double scale = 1e-9 * (1.0 + std::fabs(In[0]) + std::fabs(In[4]) + std::fabs(In[8]));
    if (mass > 0.0) {
        for (int k = 0; k < 3; k++)
            if (std::fabs(com[k] / mass) > 1e-9) {
                set_err(s, "LJ-site masses must put the centre of mass at the origin");
                return MD_ERR_ARG;
            }
        if (std::fabs(In[1]) > scale || std::fabs(In[2]) > scale || std::fabs(In[5]) > scale) {
            set_err(s, "body frame must be the principal-axes frame (off-diagonal inertia)");
            return MD_ERR_ARG;
        }
    }
    m.S = (int)sites.size();
    int na = 0, rot = 0;
    for (int a = 0; a < m.S; a++) {
        const HSite &h = sites[a];
        m.roles[a] = h.roles;
        m.lj_type[a] = (h.roles & ROLE_LJ) ? h.lj_type : 0;
        m.chg[a] = (float)h.q;
        m.mu[a] = (float)h.mu;
        m.Q[a] = (float)h.Q;
        for (int k = 0; k < 3; k++) {
            m.body[a][k] = (float)h.pos[k];
            m.axis[a][k] = (float)h.axis[k];
        }
        m.axis_slot[a] = h.has_axis ? na++ : -1;
    }
    m.NA = na;
    for (int a = m.S; a < MD_MAX_SITES; a++) m.axis_slot[a] = -1;
    for (int a = 0; a < T; a++)
        for (int b = 0; b < T; b++) {
            double xi = t->xi ? t->xi[a * T + b] : 1.0, eta = t->eta ? t->eta[a * T + b] : 1.0;
            double eps = xi * std::sqrt(t->eps[a] * t->eps[b]);
            double sig = eta * 0.5 * (t->sigma[a] + t->sigma[b]);
            m.eps4[a][b] = (float)(4.0 * eps);
            m.eps24[a][b] = (float)(24.0 * eps);
            m.sig2[a][b] = (float)(sig * sig);
            double sc6 = std::pow(sig / rc, 6.0);
            m.ushift[a][b] = lj_shift ? (float)(4.0 * eps * (sc6 * sc6 - sc6)) : 0.0f;
            m.isig[a][b] = (float)(1.0 / sig);
            m.ushift_e[a][b] = lj_shift ? (float)(4.0 * (sc6 * sc6 - sc6)) : 0.0f;
            m.dshift_s[a][b] = lj_shift ? (float)(4.0 / sig * (12.0 * sc6 * sc6 - 6.0 * sc6)) : 0.0f;
        }
    s->ent_param.clear();
    s->ent_strength.clear();
    s->lj_site_type.clear();
    for (int a = 0; a < m.S; a++) {
        const int order[3] = {ROLE_CHG, ROLE_DIP, ROLE_QUAD};
        for (int t = 0; t < 3; t++)
            if (sites[a].roles & order[t]) {
                s->ent_param.push_back(site_param[a][t]);
                s->ent_strength.push_back(t == 0 ? sites[a].q : (t == 1 ? sites[a].mu : sites[a].Q));
            }
        if (sites[a].roles & ROLE_LJ) s->lj_site_type.push_back(sites[a].lj_type);
    }
    double f = std::isinf(eps_rf) ? 1.0 : 2.0 * (eps_rf - 1.0) / (2.0 * eps_rf + 1.0);
    m.frf = (float)(f / (rc * rc * rc));
    s->n_lj = c.n_lj;
    s->n_el = c.n_chg + c.n_dip + c.n_quad;
    m.site_pairs_per_mol_pair = s->n_lj * s->n_lj + s->n_el * s->n_el;
    m.single_lj_at_com = (m.S == 1 && m.roles[0] == ROLE_LJ && sites[0].pos[0] == 0.0 && sites[0].pos[1] == 0.0 &&
                          sites[0].pos[2] == 0.0);
    m.linear = !m.single_lj_at_com;
    for (int a = 0; a < m.S; a++) {
        const HSite &h = sites[a];
        if (h.pos[0] != 0.0 || h.pos[1] != 0.0) m.linear = 0;
        if (h.has_axis && (h.axis[0] != 0.0 || h.axis[1] != 0.0 || std::fabs(std::fabs(h.axis[2]) - 1.0) > 1e-12))
            m.linear = 0;
    }
    m.mass = mass;
    for (int k = 0; k < 3; k++) {
        m.I[k] = In[4 * k];
        m.Iinv[k] = In[4 * k] > 1e-12 ? 1.0 / In[4 * k] : 0.0;
        rot += In[4 * k] > 1e-12 ? 1 : 0;
    }
    m.rot_dof = rot;
    // long-range correction (§3): U_LRC = 2 pi N^2/V sum_ab 4 eps_ab [s^12/(9 rc^9) - s^6/(3 rc^3)]
    double rc3 = rc * rc * rc, rc9 = rc3 * rc3 * rc3, cu = 0.0, cw = 0.0;
    for (int a = 0; a < c.n_lj; a++)
        for (int b = 0; b < c.n_lj; b++) {
            int ta = c.lj_type[a], tb = c.lj_type[b];
            double xi = t->xi ? t->xi[ta * T + tb] : 1.0, eta = t->eta ? t->eta[ta * T + tb] : 1.0;
            double eps = xi * std::sqrt(t->eps[ta] * t->eps[tb]);
            double sig = eta * 0.5 * (t->sigma[ta] + t->sigma[tb]);
            double s6 = std::pow(sig, 6.0), s12 = s6 * s6;
            cu += 4.0 * eps * (s12 / (9.0 * rc9) - s6 / (3.0 * rc3));
            cw += 4.0 * eps * (4.0 * s12 / (3.0 * rc9) - 2.0 * s6 / rc3);
        }
    s->lrc_u_coef = 2.0 * M_PI * cu;
    s->lrc_w_coef = 2.0 * M_PI * cw;
    double M[3] = {0, 0, 0};
    for (int a = 0; a < c.n_dip; a++) {
        const double *e = &c.dip_axis[3 * a];
        double n = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        for (int k = 0; k < 3; k++) M[k] += c.dip_mu[a] * e[k] / n;
    }
    s->rf_self_per_mol = -0.5 * f * (M[0] * M[0] + M[1] * M[1] + M[2] * M[2]) / rc3;
    return MD_OK;
}

// Keeps an editable copy of the caller's model (md_set_params replaces its
// parameters and recompiles).
md_status copy_model(md_system *s, const md_site_types *t)
{
    if (!t || t->n_comp != 1 || !t->comp) {
        set_err(s, "md_site_types: exactly one component is supported (got %d)", t ? t->n_comp : -1);
        return (t && t->n_comp > 1) ? MD_ERR_UNSUPPORTED : MD_ERR_ARG;
    }
    const md_component &c = t->comp[0];
    if (t->n_types < 0 || t->n_types > MD_MAX_TYPES || (t->n_types > 0 && (!t->eps || !t->sigma)) || c.n_lj < 0 ||
        c.n_chg < 0 || c.n_dip < 0 || c.n_quad < 0 || (c.n_lj && (!c.lj_pos || !c.lj_type || !c.lj_mass)) ||
        (c.n_chg && (!c.chg_pos || !c.chg_q)) || (c.n_dip && (!c.dip_pos || !c.dip_axis || !c.dip_mu)) ||
        (c.n_quad && (!c.quad_pos || !c.quad_axis || !c.quad_Q))) {
        set_err(s, "md_site_types / md_component: bad count or NULL array");
        return t->n_types > MD_MAX_TYPES ? MD_ERR_UNSUPPORTED : MD_ERR_ARG;
    }
    HostModel &h = s->hm;
    const int T = t->n_types;
    h.T = T;
    h.eps.assign(t->eps, t->eps + T);
    h.sigma.assign(t->sigma, t->sigma + T);
    h.has_xi = t->xi != nullptr;
    h.has_eta = t->eta != nullptr;
    h.xi.assign(T * T, 1.0);
    h.eta.assign(T * T, 1.0);
    if (t->xi) h.xi.assign(t->xi, t->xi + T * T);
    if (t->eta) h.eta.assign(t->eta, t->eta + T * T);
    h.n_lj = c.n_lj;
    h.n_chg = c.n_chg;
    h.n_dip = c.n_dip;
    h.n_quad = c.n_quad;
    auto cp = [](std::vector<double> &v, const double *p, int n) { v.assign(p ? p : nullptr, p ? p + n : nullptr); };
    cp(h.lj_pos, c.lj_pos, 3 * c.n_lj);
    cp(h.lj_mass, c.lj_mass, c.n_lj);
    h.lj_type.assign(c.lj_type ? c.lj_type : nullptr, c.lj_type ? c.lj_type + c.n_lj : nullptr);
    cp(h.chg_pos, c.chg_pos, 3 * c.n_chg);
    cp(h.chg_q, c.chg_q, c.n_chg);
    cp(h.dip_pos, c.dip_pos, 3 * c.n_dip);
    cp(h.dip_axis, c.dip_axis, 3 * c.n_dip);
    cp(h.dip_mu, c.dip_mu, c.n_dip);
    cp(h.quad_pos, c.quad_pos, 3 * c.n_quad);
    cp(h.quad_axis, c.quad_axis, 3 * c.n_quad);
    cp(h.quad_Q, c.quad_Q, c.n_quad);
    h.view();
    return MD_OK;
}

md_status alloc_molecules(md_system *s, long long n)
{
    DevState &d = s->d;
    if (n <= s->cap && d.r != nullptr) {
        d.n = n;
        return MD_OK;
    }
    double **dbl[] = {&d.r, &d.v, &d.j, &d.r2, &d.v2, &d.j2, &d.F, &d.tau};
    for (auto p : dbl) {
        cudaFree(*p);
        *p = nullptr;
    }
    cudaFree(d.q);
    cudaFree(d.q2);
    cudaFree(d.ids);
    cudaFree(d.ids2);
    cudaFree(d.cell);
    cudaFree(d.perm);
    cudaFree(d.perm2);
    cudaFree(d.com);
    cudaFree(d.geo);
    cudaFree(d.facc);
    d.facc = nullptr;
    d.q = d.q2 = nullptr;
    d.ids = d.ids2 = d.cell = d.perm = d.perm2 = nullptr;
    d.com = d.geo = nullptr;
    s->cap = 0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    cudaError_t e = cudaSuccess;
    for (auto p : dbl)
        if (e == cudaSuccess) e = cudaMalloc((void **)p, nn * 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.q, nn * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.q2, nn * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.ids, nn * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.ids2, nn * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.cell, nn * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.perm, nn * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.perm2, nn * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.com, nn * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.geo, nn * (size_t)(d.K > 0 ? d.K : 1) * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.facc, nn * FACC_STRIDE * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(s, e, "allocating molecule buffers");
    s->cap = n;
    d.n = n;
    return MD_OK;
}

void drop_step_graphs(md_system *s)
{
    for (int p = 0; p < 2; p++)
        if (s->gexec[p]) {
            cudaGraphExecDestroy(s->gexec[p]);
            s->gexec[p] = nullptr;
        }
}

void free_all(md_system *s)
{
    drop_step_graphs(s);
    DevState &d = s->d;
    void *ptrs[] = {d.r, d.v, d.q, d.j, d.r2, d.v2, d.q2, d.j2, d.ids, d.ids2, d.F, d.tau, d.cell, d.cell_count,
                    d.cell_start, d.cell_fill, d.perm, d.perm2, d.com, d.geo, d.scan_tmp, d.partials,
                    d.kin_partials, d.thermo, d.flags, d.facc, s->adj_partials};
    for (void *p : ptrs) cudaFree(p);
    for (auto &p : s->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : s->pool) cudaEventDestroy(e);
}

md_status check_flags(md_system *s)
{
    int h[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(h, s->d.flags, sizeof h, cudaMemcpyDeviceToHost), "reading device flags");
    if (h[FLAG_NONFINITE]) {
        set_err(s, "non-finite force, torque or position detected on the device");
        return MD_ERR_NONFINITE;
    }
    if (h[FLAG_OVERFLOW]) {
        set_err(s, "a fixed-capacity device buffer overflowed");
        return MD_ERR_OVERFLOW;
    }
    if (h[FLAG_TIMEOUT]) {
        set_err(s, "a bounded device wait gave up");
        return MD_ERR_TIMEOUT;
    }
    if (h[FLAG_INPUT]) {
        set_err(s, "md_set_molecules (device input): non-finite r, v or j, or a zero or non-finite quaternion");
        return MD_ERR_NONFINITE;
    }
    return MD_OK;
}

md_status do_rebuild(md_system *s, cudaStream_t st, bool need_cellid, const double *beta = nullptr)
{
    TimeScope ts(s, st, 1);
    if (need_cellid) CK(launch_cellid(s->g, s->d, st), "cell id kernel");
    CK(launch_rebuild(s->g, s->m, s->d, st, beta, s->opt.deterministic, s->half_eff), "cell rebuild kernels");
    s->binned = true;
    s->acc_zeroed = s->half_eff && !s->opt.deterministic && s->d.n > 0;
    return MD_OK;
}

md_status do_force(md_system *s, cudaStream_t st)
{
    TimeScope ts(s, st, 3);
    // cells in counter order unless the energy sums must group identically on every launch
    CK(launch_force(s->g, s->m, s->d, s->half_eff, !s->opt.deterministic, s->n_force_blocks, st, s->acc_zeroed),
       "force kernel");
    s->acc_zeroed = false;
    s->forces_valid = true;
    s->f_in_acc = s->half_eff != 0;
    return MD_OK;
}

// One leapfrog step (§3) on stream st: integrate (+ NVT factor, §2) ->
// rebuild (the factor applied in the reorder) -> forces.  The integrator
// reads the forces where the force kernel leaves them: the FP32 records in
// the half shell, the FP64 arrays in the full shell.
md_status one_step(md_system *s, double dt, double T_target, cudaStream_t st)
{
    const bool nvt = T_target > 0.0;
    const double dof = 3.0 * (double)s->d.n - 3.0 + (double)s->m.rot_dof * (double)s->d.n;
    const bool thermo = nvt && dof > 0.0 && s->d.n > 0;
    {
        TimeScope ts(s, st, 0);
        // a non-deterministic rebuild leaves the histogram at zero
        CK(launch_integrate(s->g, s->m, s->d, dt, s->half_eff, st, s->opt.deterministic), "integrate kernel");
        if (thermo) CK(launch_thermostat(s->m, s->d, s->n_kin_blocks, T_target, dof, st), "thermostat kernels");
    }
    md_status ms = do_rebuild(s, st, false, thermo ? s->d.thermo : nullptr);
    if (ms != MD_OK) return ms;
    return do_force(s, st);
}

// FP64 F and tau for the callers that read them (observables, md_get_forces):
// the integrator reads the FP32 accumulators directly, so the conversion
// runs only when something outside the step needs it.
md_status forces_to_f64(md_system *s, cudaStream_t st)
{
    if (!s->f_in_acc) return MD_OK;
    TimeScope ts(s, st, 7);
    CK(launch_force_finalize(s->d, st), "force finalize kernel");
    s->f_in_acc = false;
    return MD_OK;
}

}  // namespace

void model_info(const md_system *s, ModelInfo *out)
{
    out->m = s->m;
    out->g = s->g;
    out->lrc_u_coef = s->lrc_u_coef;
    out->lrc_w_coef = s->lrc_w_coef;
    out->rf_self_per_mol = s->rf_self_per_mol;
}

extern "C" {

const char *md_status_str(md_status st)
{
    switch (st) {
    case MD_OK: return "MD_OK";
    case MD_ERR_ARG: return "MD_ERR_ARG: invalid argument";
    case MD_ERR_BOX: return "MD_ERR_BOX: box edge smaller than twice the cut-off";
    case MD_ERR_STATE: return "MD_ERR_STATE: call out of order";
    case MD_ERR_CUDA: return "MD_ERR_CUDA: CUDA runtime error";
    case MD_ERR_OOM: return "MD_ERR_OOM: device allocation failed";
    case MD_ERR_NONFINITE: return "MD_ERR_NONFINITE: non-finite value detected";
    case MD_ERR_OVERFLOW: return "MD_ERR_OVERFLOW: buffer capacity exceeded";
    case MD_ERR_TIMEOUT: return "MD_ERR_TIMEOUT: bounded device wait gave up";
    case MD_ERR_UNSUPPORTED: return "MD_ERR_UNSUPPORTED: input outside what the library supports";
    }
    return "unknown md_status";
}

const char *md_last_error(const md_system *s) { return s ? s->err : "NULL handle"; }

md_status md_create(const double box[3], double cutoff, const md_site_types *types, const md_options *options,
                    md_system **out)
{
    if (!out || !box || !types) return MD_ERR_ARG;
    *out = nullptr;
    if (!(std::isfinite(cutoff) && cutoff > 0.0) || !finite3(box) || !(box[0] > 0 && box[1] > 0 && box[2] > 0))
        return MD_ERR_ARG;
    for (int k = 0; k < 3; k++)
        if (box[k] < 2.0 * cutoff) return MD_ERR_BOX;
    md_options opt = {INFINITY, 0, 0, 1, 0, 1};
    if (options) opt = *options;
    if (std::isnan(opt.eps_rf) || (!std::isinf(opt.eps_rf) && opt.eps_rf < 1.0) || (std::isinf(opt.eps_rf) && opt.eps_rf < 0))
        return MD_ERR_ARG;
    if (opt.cell_div == 0) opt.cell_div = 1;
    if (opt.cell_div != 1 && opt.cell_div != 2) return MD_ERR_ARG;
    md_system *s = new (std::nothrow) md_system();
    if (!s) return MD_ERR_OOM;
    s->opt = opt;
    s->rc = cutoff;
    md_status st = copy_model(s, types);
    if (st == MD_OK) st = compile_model(s, &s->hm.types, cutoff, opt.lj_shift, opt.eps_rf);
    if (st != MD_OK) {
        delete s;
        return st;
    }
    Grid &g = s->g;
    g.m = opt.cell_div;  // stencil radius in cells
    long long ncell = 1;
    for (int k = 0; k < 3; k++) {
        // edge >= cutoff / m: the stencil's m cells per side cover the cut-off
        const double nd = std::floor(box[k] * g.m / (cutoff * (1.0 + 1e-9)));
        if (nd > 2e9) {
            delete s;
            return MD_ERR_UNSUPPORTED;
        }
        int nc = (int)nd;
        g.nc[k] = nc < 1 ? 1 : nc;
        g.L[k] = box[k];
        g.ell[k] = box[k] / g.nc[k];
        g.iell[k] = 1.0 / g.ell[k];
        g.ellf[k] = (float)g.ell[k];
        ncell *= g.nc[k];
    }
    if (ncell > (1LL << 31) - 2) {
        delete s;
        return MD_ERR_UNSUPPORTED;
    }
    g.ncell = ncell;
    g.rc2 = cutoff * cutoff;
    g.rc2f = (float)g.rc2;
    g.bandf = (float)(2e-5 * g.rc2);
    // the half stencil counts each pair once only if its cells are distinct
    const int nmin = 2 * g.m + 1;
    s->half_eff = (opt.half_shell && !opt.deterministic && g.nc[0] >= nmin && g.nc[1] >= nmin && g.nc[2] >= nmin) ? 1 : 0;
    s->d.K = s->m.single_lj_at_com ? 0 : (s->m.linear ? 1 : s->m.S + s->m.NA);

    // upper bound of the force grid: one block per MD_WARPS units of work, a
    // cell being split into up to 4 units in small systems
    long long fb = (4 * ncell + MD_WARPS - 1) / MD_WARPS;
    s->n_force_blocks = (int)(fb < force_blocks_default() ? fb : force_blocks_default());
    s->n_kin_blocks = device_sms() * 4;
    DevState &d = s->d;
    cudaError_t e = cudaMalloc((void **)&d.cell_count, sizeof(int) * ncell);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.cell_start, sizeof(int) * (ncell + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.cell_fill, sizeof(int) * ncell);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.scan_tmp, sizeof(int) * (scan_blocks(ncell) + 1));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.partials, sizeof(double) * (P_COUNT * (size_t)s->n_force_blocks + 1));
    d.cell_ctr = e == cudaSuccess ? reinterpret_cast<unsigned *>(d.partials + P_COUNT * (size_t)s->n_force_blocks) : nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.kin_partials, sizeof(double) * 4 * s->n_kin_blocks);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.thermo, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d.flags, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(d.flags, 0, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(d.cell_start, 0, sizeof(int) * (ncell + 1));
    if (e != cudaSuccess) {
        md_status r = cuda_fail(s, e, "md_create allocations");
        free_all(s);
        delete s;
        return r;
    }
    *out = s;
    return MD_OK;
}

void md_destroy(md_system *s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    free_all(s);
    delete s;
}

int64_t md_n_molecules(const md_system *s) { return s ? (int64_t)s->d.n : -1; }

md_status md_set_molecules(md_system *s, int64_t n, const int32_t *comp_id, const double *r, const double *v,
                           const double *q, const double *j, int32_t on_device, void *cuda_stream)
{
    if (!s) return MD_ERR_ARG;
    if (n < 0 || n > (1LL << 31) - 1 || (n > 0 && (!r || !q))) {
        set_err(s, "md_set_molecules: n out of range or NULL r/q");
        return MD_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (comp_id) {
        if (on_device) {
            set_err(s, "md_set_molecules: device comp_id is not supported (single component)");
            return MD_ERR_UNSUPPORTED;
        }
        for (int64_t i = 0; i < n; i++)
            if (comp_id[i] != 0) {
                set_err(s, "md_set_molecules: comp_id %d out of range", comp_id[i]);
                return MD_ERR_ARG;
            }
    }
    // values are validated on the device by the preparation kernel (one
    // pass over the copied state instead of a host scan of the input)
    drop_step_graphs(s);
    s->parity = 0;
    md_status ms = alloc_molecules(s, n);
    if (ms != MD_OK) return ms;
    DevState &d = s->d;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t b3 = sizeof(double) * 3 * (size_t)n, b4 = sizeof(double) * 4 * (size_t)n;
    if (n > 0) {
        CK(cudaMemcpyAsync(d.r, r, b3, kind, st), "copy r");
        CK(cudaMemcpyAsync(d.q, q, b4, kind, st), "copy q");
        if (v) CK(cudaMemcpyAsync(d.v, v, b3, kind, st), "copy v");
        else CK(cudaMemsetAsync(d.v, 0, b3, st), "zero v");
        if (j) CK(cudaMemcpyAsync(d.j, j, b3, kind, st), "copy j");
        else CK(cudaMemsetAsync(d.j, 0, b3, st), "zero j");
        CK(cudaMemsetAsync(d.F, 0, b3, st), "zero F");
        CK(cudaMemsetAsync(d.tau, 0, b3, st), "zero tau");
    }
    CK(cudaMemsetAsync(d.flags + FLAG_INPUT, 0, sizeof(int), st), "clear input flag");
    CK(launch_prepare_input(s->g, d, st), "input preparation kernel");
    s->has_mol = true;
    s->binned = false;
    s->forces_valid = false;
    s->f_in_acc = false;
    s->dt_last = 0.0;
    s->time = 0.0;
    s->step = 0;
    s->last_stream = st;
    ms = do_rebuild(s, st, true);
    if (ms != MD_OK) return ms;
    if (!on_device) {
        int bad = 0;  // read on the stream: one wait for the copies, the kernels and the flag
        CK(cudaMemcpyAsync(&bad, d.flags + FLAG_INPUT, sizeof bad, cudaMemcpyDeviceToHost, st), "reading the input flag");
        CK(cudaStreamSynchronize(st), "md_set_molecules sync");
        if (bad) {
            CK(cudaMemset(d.flags + FLAG_INPUT, 0, sizeof(int)), "clear input flag");
            s->has_mol = false;
            set_err(s, "md_set_molecules: non-finite r, v or j, or a zero or non-finite quaternion");
            return MD_ERR_ARG;
        }
    }
    return MD_OK;
}

md_status md_compute_forces(md_system *s, void *cuda_stream)
{
    if (!s) return MD_ERR_ARG;
    if (!s->has_mol) {
        set_err(s, "md_compute_forces: call md_set_molecules first");
        return MD_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->last_stream = st;
    if (!s->binned) {
        md_status ms = do_rebuild(s, st, true);
        if (ms != MD_OK) return ms;
    }
    return do_force(s, st);
}

md_status md_step(md_system *s, int32_t n_steps, double dt, double T_target, void *cuda_stream)
{
    if (!s) return MD_ERR_ARG;
    if (n_steps < 0 || !std::isfinite(dt) || !(dt > 0.0) || !std::isfinite(T_target)) {
        set_err(s, "md_step: n_steps >= 0, finite dt > 0 and finite T_target required");
        return MD_ERR_ARG;
    }
    if (!s->has_mol) {
        set_err(s, "md_step: call md_set_molecules first");
        return MD_ERR_STATE;
    }
    if (!(s->m.mass > 0.0)) {
        set_err(s, "md_step: the component has no mass");
        return MD_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    s->last_stream = st;
    if (!s->forces_valid) {
        md_status ms = md_compute_forces(s, st);
        if (ms != MD_OK) return ms;
    }
    int k = 0;
    if (!s->profiling && n_steps >= 2 && s->d.n > 0) {
        // pairs of steps as replays of a captured graph (the buffer assignment
        // is back where it started after two steps)
        for (; k + 2 <= n_steps; k += 2) {
            const int p = s->parity;
            if (!s->gexec[p] || s->gdt[p] != dt || s->gT[p] != T_target) {
                if (s->gexec[p]) cudaGraphExecDestroy(s->gexec[p]);
                s->gexec[p] = nullptr;
                cudaStream_t cs;
                CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
                cudaGraph_t graph;
                cudaError_t eb = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                if (eb != cudaSuccess) {
                    cudaStreamDestroy(cs);
                    CK(eb, "begin capture");
                }
                const DevState saved = s->d;
                md_status ms = one_step(s, dt, T_target, cs);
                if (ms == MD_OK) ms = one_step(s, dt, T_target, cs);
                const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
                s->d = saved;  // captured, not run: the state has not moved
                cudaStreamDestroy(cs);
                if (ms != MD_OK) {
                    if (ec == cudaSuccess) cudaGraphDestroy(graph);
                    return ms;
                }
                CK(ec, "end capture");
                const cudaError_t ei = cudaGraphInstantiate(&s->gexec[p], graph, 0);
                cudaGraphDestroy(graph);
                CK(ei, "graph instantiate");
                s->gdt[p] = dt;
                s->gT[p] = T_target;
            }
            CK(cudaGraphLaunch(s->gexec[p], st), "graph launch");
            s->forces_valid = true;
            s->f_in_acc = s->half_eff != 0;
            s->step += 2;
            s->time += 2.0 * dt;
        }
    }
    for (; k < n_steps; k++) {
        md_status ms = one_step(s, dt, T_target, st);
        if (ms != MD_OK) return ms;
        s->parity ^= 1;
        s->step++;
        s->time += dt;
    }
    s->dt_last = dt;
    return MD_OK;
}

md_status md_sync(md_system *s, void *cuda_stream)
{
    if (!s) return MD_ERR_ARG;
    md_status mf = forces_to_f64(s, (cudaStream_t)cuda_stream);  // also checks the latest forces for non-finite values
    if (mf != MD_OK) return mf;
    CK(cudaStreamSynchronize((cudaStream_t)cuda_stream), "stream synchronize");
    if (s->profiling) drain_timings(s);
    return check_flags(s);
}

md_status md_energy_virial(md_system *s, md_observables *out)
{
    if (!s || !out) return MD_ERR_ARG;
    if (!s->forces_valid) {
        set_err(s, "md_energy_virial: no force evaluation yet");
        return MD_ERR_STATE;
    }
    cudaStream_t st = s->last_stream;
    md_status mf = forces_to_f64(s, st);
    if (mf != MD_OK) return mf;
    {
        TimeScope ts(s, st, 4);
        CK(launch_kinetic(s->m, s->d, 0.5 * s->dt_last, s->n_kin_blocks, st), "kinetic kernel");
    }
    std::vector<double> fp((size_t)P_COUNT * s->n_force_blocks), kp((size_t)4 * s->n_kin_blocks);
    CK(cudaMemcpyAsync(fp.data(), s->d.partials, fp.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "copy partials");
    CK(cudaMemcpyAsync(kp.data(), s->d.kin_partials, kp.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
       "copy kinetic partials");
    CK(cudaStreamSynchronize(st), "md_energy_virial sync");
    if (s->profiling) drain_timings(s);
    md_status fl = check_flags(s);
    double acc[P_COUNT] = {0};
    for (int b = 0; b < s->n_force_blocks; b++)
        for (int k = 0; k < P_COUNT; k++) acc[k] += fp[(size_t)b * P_COUNT + k];
    double kt = 0.0, kr = 0.0;
    for (int b = 0; b < s->n_kin_blocks; b++) {
        kt += kp[4 * b];
        kr += kp[4 * b + 1];
    }
    memset(out, 0, sizeof *out);
    const double N = (double)s->d.n, V = s->g.L[0] * s->g.L[1] * s->g.L[2];
    out->U_pot = acc[P_U];
    out->W = acc[P_W];
    out->W_xx = acc[P_WXX];
    out->W_yy = acc[P_WYY];
    out->W_zz = acc[P_WZZ];
    out->n_mol_pairs = (int64_t)llround(acc[P_NMOL]);
    out->n_site_pairs = (int64_t)llround(acc[P_NSITE]);
    out->n_examined = (int64_t)llround(acc[P_NEXAM]);
    out->U_lrc = s->opt.lj_lrc ? s->lrc_u_coef * N * N / V : 0.0;
    out->W_lrc = s->opt.lj_lrc ? s->lrc_w_coef * N * N / V : 0.0;
    out->U_rf_self = s->rf_self_per_mol * N;
    out->K_trans = kt;
    out->K_rot = kr;
    double dof = 3.0 * N - 3.0 + (double)s->m.rot_dof * N;
    out->T = dof > 0 ? 2.0 * (kt + kr) / dof : 0.0;
    out->P = (2.0 * kt + out->W + out->W_lrc) / (3.0 * V);
    out->time = s->time;
    out->step = s->step;
    out->n_molecules = (int64_t)s->d.n;
    return fl;
}

md_status md_get_molecules(md_system *s, double *r, double *v, double *q, double *j, int32_t on_device,
                           void *cuda_stream)
{
    if (!s) return MD_ERR_ARG;
    if (!s->has_mol) {
        set_err(s, "md_get_molecules: call md_set_molecules first");
        return MD_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    DevState &d = s->d;
    double *dst[4] = {r, v, q, j};
    double *tmp[4] = {d.r2, d.v2, d.q2, d.j2};
    const int w[4] = {3, 3, 4, 3};
    double *target[4];
    for (int k = 0; k < 4; k++) target[k] = !dst[k] ? nullptr : (on_device ? dst[k] : tmp[k]);
    if (d.n > 0) {
        // one kernel for the four arrays, then the copies back to back
        CK(launch_scatter_state(d, target[0], target[1], target[2], target[3], st), "scatter kernel");
        if (!on_device)
            for (int k = 0; k < 4; k++)
                if (dst[k])
                    CK(cudaMemcpyAsync(dst[k], tmp[k], sizeof(double) * w[k] * (size_t)d.n, cudaMemcpyDeviceToHost,
                                       st),
                       "copy state to host");
    }
    CK(cudaStreamSynchronize(st), "md_get_molecules sync");
    return check_flags(s);
}

md_status md_get_forces(md_system *s, double *F, double *tau, int32_t on_device, void *cuda_stream)
{
    if (!s) return MD_ERR_ARG;
    if (!s->forces_valid) {
        set_err(s, "md_get_forces: no force evaluation yet");
        return MD_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    md_status mf = forces_to_f64(s, st);
    if (mf != MD_OK) return mf;
    DevState &d = s->d;
    const double *src[2] = {d.F, d.tau};
    double *dst[2] = {F, tau};
    double *tmp[2] = {d.r2, d.v2};
    for (int k = 0; k < 2; k++) {
        if (!dst[k] || d.n == 0) continue;
        double *target = on_device ? dst[k] : tmp[k];
        CK(launch_scatter_out(d, src[k], 3, target, st), "scatter kernel");
        if (!on_device)
            CK(cudaMemcpyAsync(dst[k], tmp[k], sizeof(double) * 3 * (size_t)d.n, cudaMemcpyDeviceToHost, st),
               "copy forces to host");
    }
    CK(cudaStreamSynchronize(st), "md_get_forces sync");
    return check_flags(s);
}

int32_t md_n_params(const md_system *s)
{
    if (!s) return -1;
    const HostModel &h = s->hm;
    return 2 * h.T + h.n_chg + h.n_dip + h.n_quad;
}

md_status md_get_params(md_system *s, double *theta)
{
    if (!s || !theta) return MD_ERR_ARG;
    const HostModel &h = s->hm;
    int k = 0;
    for (int t = 0; t < h.T; t++) theta[k++] = h.eps[t];
    for (int t = 0; t < h.T; t++) theta[k++] = h.sigma[t];
    for (int a = 0; a < h.n_chg; a++) theta[k++] = h.chg_q[a];
    for (int a = 0; a < h.n_dip; a++) theta[k++] = h.dip_mu[a];
    for (int a = 0; a < h.n_quad; a++) theta[k++] = h.quad_Q[a];
    return MD_OK;
}

md_status md_set_params(md_system *s, const double *theta, int32_t n_params)
{
    if (!s || !theta) return MD_ERR_ARG;
    drop_step_graphs(s);  // the model is a captured kernel argument
    if (n_params != md_n_params(s)) {
        set_err(s, "md_set_params: expected %d parameters, got %d", md_n_params(s), n_params);
        return MD_ERR_ARG;
    }
    HostModel h = s->hm;
    int k = 0;
    for (int t = 0; t < h.T; t++) h.eps[t] = theta[k++];
    for (int t = 0; t < h.T; t++) h.sigma[t] = theta[k++];
    for (int a = 0; a < h.n_chg; a++) h.chg_q[a] = theta[k++];
    for (int a = 0; a < h.n_dip; a++) h.dip_mu[a] = theta[k++];
    for (int a = 0; a < h.n_quad; a++) h.quad_Q[a] = theta[k++];
    h.view();
    DevModel keep = s->m;
    md_status st = compile_model(s, &h.types, s->rc, s->opt.lj_shift, s->opt.eps_rf);
    if (st != MD_OK) {
        s->m = keep;
        compile_model(s, &s->hm.types, s->rc, s->opt.lj_shift, s->opt.eps_rf);
        return st;
    }
    s->hm = h;
    s->hm.view();
    s->forces_valid = false;
    return MD_OK;
}

md_status md_param_grad(md_system *s, int32_t n_cfg, int64_t n, const double *r_all, const double *q_all,
                        int32_t on_device, double *dU, double *dW, double *means, void *cuda_stream)
{
    if (!s || n_cfg < 1 || n < 0 || (n > 0 && (!r_all || !q_all)) || !dU || !dW || !means) return MD_ERR_ARG;
    const int nacc = adjoint_nacc(s->m);
    if (nacc < 0) {
        set_err(s, "md_param_grad: the adjoint kernel is compiled for the built-in site signatures only");
        return MD_ERR_UNSUPPORTED;
    }
    if (s->g.m != 1) {
        set_err(s, "md_param_grad: the adjoint kernel traverses cells of edge >= cutoff (cell_div 1) only");
        return MD_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (s->adj_nacc != nacc) {
        cudaFree(s->adj_partials);
        s->adj_partials = nullptr;
        s->adj_nacc = 0;
        CK(cudaMalloc((void **)&s->adj_partials, sizeof(double) * (size_t)nacc * s->n_force_blocks),
           "allocating adjoint partials");
        s->adj_nacc = nacc;
    }
    const int half = (s->g.nc[0] >= 3 && s->g.nc[1] >= 3 && s->g.nc[2] >= 3) ? 1 : 0;
    std::vector<double> tot(nacc, 0.0), part((size_t)nacc * s->n_force_blocks);
    for (int c = 0; c < n_cfg; c++) {
        md_status ms = md_set_molecules(s, n, nullptr, r_all + (size_t)c * n * 3, nullptr, q_all + (size_t)c * n * 4,
                                        nullptr, on_device, cuda_stream);
        if (ms != MD_OK) return ms;
        {
            TimeScope ts(s, st, 6);
            CK(launch_adjoint(s->g, s->m, s->d, half, !s->opt.deterministic, s->n_force_blocks, s->adj_partials,
                              nacc, st),
               "adjoint kernel");
        }
        CK(cudaMemcpyAsync(part.data(), s->adj_partials, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
           "copy adjoint partials");
        CK(cudaStreamSynchronize(st), "md_param_grad sync");
        for (int b = 0; b < s->n_force_blocks; b++)
            for (int q = 0; q < nacc; q++) tot[q] += part[(size_t)b * nacc + q];
    }
    if (s->profiling) drain_timings(s);
    for (auto &v : tot) v /= (double)n_cfg;
    const HostModel &h = s->hm;
    const int T = h.T, P = md_n_params(s);
    for (int p = 0; p < P; p++) dU[p] = dW[p] = 0.0;
    auto mix = [&](int ta, int tb, double &eps, double &sig, double &eta) {
        eps = h.xi[ta * T + tb] * std::sqrt(h.eps[ta] * h.eps[tb]);
        eta = h.eta[ta * T + tb];
        sig = eta * 0.5 * (h.sigma[ta] + h.sigma[tb]);
    };
    // chain rule through Lorentz-Berthelot: d eps_ab / d eps_t = eps_ab (n_t) / (2 eps_t),
    // d sigma_ab / d sigma_t = eta_ab n_t / 2, n_t = [a is t] + [b is t]
    auto lj_chain = [&](int ta, int tb, double su_e, double sw_e, double su_s, double sw_s) {
        double eps, sig, eta;
        mix(ta, tb, eps, sig, eta);
        for (int t = 0; t < T; t++) {
            const double nt = (double)((ta == t) + (tb == t));
            if (nt == 0.0) continue;
            const double de = h.eps[t] > 0.0 ? eps * nt / (2.0 * h.eps[t]) : 0.0;
            const double ds = eta * nt * 0.5;
            dU[t] += su_e * de;
            dW[t] += sw_e * de;
            dU[T + t] += su_s * ds;
            dW[T + t] += sw_s * ds;
        }
    };
    const int NLJ = (int)s->lj_site_type.size(), NE = (int)s->ent_param.size();
    for (int a = 0; a < NLJ; a++)
        for (int b = 0; b < NLJ; b++) {
            const double *v = &tot[4 * (a * NLJ + b)];
            lj_chain(s->lj_site_type[a], s->lj_site_type[b], v[0], v[1], v[2], v[3]);
        }
    // bilinear in the strengths
    for (int ea = 0; ea < NE; ea++)
        for (int eb = 0; eb < NE; eb++) {
            const double U1 = tot[4 * NLJ * NLJ + 2 * (ea * NE + eb)], W1 = tot[4 * NLJ * NLJ + 2 * (ea * NE + eb) + 1];
            dU[s->ent_param[ea]] += s->ent_strength[eb] * U1;
            dW[s->ent_param[ea]] += s->ent_strength[eb] * W1;
            dU[s->ent_param[eb]] += s->ent_strength[ea] * U1;
            dW[s->ent_param[eb]] += s->ent_strength[ea] * W1;
        }
    double U = tot[nacc - 2], W = tot[nacc - 1];
    if (s->opt.lj_lrc) {
        // isotropic tail (§3) per LJ centre pair and its parameter derivatives
        const double V = s->g.L[0] * s->g.L[1] * s->g.L[2];
        const double rc = s->rc, rc3 = rc * rc * rc, rc9 = rc3 * rc3 * rc3;
        const double pre = 2.0 * M_PI * (double)n * (double)n / V;
        for (int a = 0; a < h.n_lj; a++)
            for (int b = 0; b < h.n_lj; b++) {
                const int ta = h.lj_type[a], tb = h.lj_type[b];
                double eps, sig, eta;
                mix(ta, tb, eps, sig, eta);
                const double s5 = std::pow(sig, 5.0), s6 = s5 * sig, s11 = s6 * s5, s12 = s6 * s6;
                const double uL = 4.0 * (s12 / (9.0 * rc9) - s6 / (3.0 * rc3));
                const double wL = 4.0 * (4.0 * s12 / (3.0 * rc9) - 2.0 * s6 / rc3);
                U += pre * eps * uL;
                W += pre * eps * wL;
                lj_chain(ta, tb, pre * uL, pre * wL, pre * 4.0 * eps * (12.0 * s11 / (9.0 * rc9) - 2.0 * s5 / rc3),
                         pre * 4.0 * eps * (16.0 * s11 / rc9 - 12.0 * s5 / rc3));
            }
    }
    means[0] = U;
    means[1] = W;
    s->forces_valid = false;
    return MD_OK;
}

md_status md_profile(md_system *s, int32_t enable)
{
    if (!s) return MD_ERR_ARG;
    s->profiling = enable != 0;
    return MD_OK;
}

md_status md_kernel_times_get(md_system *s, md_kernel_times *out)
{
    if (!s || !out) return MD_ERR_ARG;
    CK(cudaStreamSynchronize(s->last_stream), "md_kernel_times_get sync");
    drain_timings(s);
    *out = s->times;
    memset(&s->times, 0, sizeof s->times);
    return MD_OK;
}

}  // extern "C"
