// C ABI: context management, the per-stage pipeline and the graph-captured RK driver.
//
// One right-hand-side evaluation (one Runge-Kutta stage) is about 12 launches on two
// streams joined before the right-hand side:
//   side stream: deriv r, theta, phi (first derivatives of 21 BSSN fields) | interface mean
//                of d_r | deriv r, theta, phi (second derivatives of 11 fields) | interface
//                mean of d_rr
//   main stream: prep | deriv r, theta, phi (flux divergence) | (join) | rhs (+ RK stage
//                combination)
// A time step adds the filter (3 directional contractions + interface mean of the BSSN
// copies).  grmhd_step records nsteps steps into one CUDA graph.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "grmhd_internal.h"
#include "host_ops.h"

using namespace gk;

// NVTX range around a public call (shown by Nsight timelines; a no-op without a tool)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct grmhd_ctx {
    grmhd_grid grid;
    grmhd_physics phys;
    grmhd_opts opts;
    Dims d;
    PhysParams pp;
    cudaStream_t stream;
    bool own_stream;
    // side stream of a stage: the BSSN derivative chain runs there while the primitive
    // recovery and the flux divergence run on `stream` (fork / join events)
    cudaStream_t s2;
    cudaEvent_t ev_fork, ev_join;
    // device buffers
    double* U[3];            // U[0] = state, U[1], U[2] = stage buffers
    double* acc;             // RK4 accumulator (allocated for integrator = 1)
    double* prim;
    double* flux;
    double* tmn;
    double* lam;
    double* d1;
    double* d2;
    double* divF;
    double* scratch;         // nv * P
    double* divB;            // d_i (sqrt(gamma) B^i) (GLM only)
    double* ham;             // Hamiltonian constraint per node (diagnostics)
    double* met;             // 9 * P: the metric of the last k_prep (e^{4phi}, e^{-4phi}, sqrt(gamma), gammatilde^ij)
    double* ham_out;         // non-null while a diagnostic stage is enqueued: k_rhs writes H there
    int nv;                  // evolved variables: GRMHD_NV, + 1 (psi) with GLM
    double* Dr;              // Nr x Nr reference CGL matrix on [-1, 1]
    double* Dt;              // Nt x Nt Gauss matrix scaled to [theta_min, theta_max]
    double* Dp;              // circulant row
    double* Fr;
    double* Ft;
    double* Fp;
    double* Ds[3];           // reflection-split derivative operators (nullptr: dense only)
    double* Fs[3];           // reflection-split filter operators
    double* r_scale;         // E
    double* wq;              // P quadrature weights
    double* hmin;            // n_inst CFL spacings
    double* dt;              // n_inst time steps
    double* diag;            // 8
    unsigned long long* nfail;
    unsigned long long* lam_bits;   // n_inst
    unsigned char* iface_dev;       // E: element e coupled to e + 1
    int* elem_inst_dev;             // E: owning instance
    int* nan_flag;
    DerivJob* jobs;          // all job lists
    // mixed-precision (tensor-core) contractions
    uint8_t* tc_img[3];      // operator images r / theta / phi
    // FP64-accurate tensor-core contractions (opts.contraction = 0): digit-slice images of
    // the derivative (radial: one per element, r-scale folded in) and filter operators
    uint8_t* fx_d[3];
    uint8_t* fx_f[3];
    long long fx_estride;    // bytes between the per-element radial derivative images
    TcJob* tcjobs;
    int tc_first[3][3];      // [buffer][dir]
    int tc_second[3];
    int* tc_err;
    int job_first[3][3];     // [buffer][dir] offset of the first-derivative jobs
    int job_first_n;
    int job_second[3];       // [dir] offset of the second-derivative jobs
    int job_second_n[3];
    int job_filter[3][3][2]; // [buffer][dir][group] offset (8 or 24 jobs)
    int job_dbg;
    // Fourier theta basis (grid.theta_basis = 1): theta contractions fold the phi pairs
    // (l, l + N_phi/2) into sums / differences, contract each half with the even or
    // odd extension operator, and unfold (kernels_deriv.cu)
    int ft;                  // 1: Fourier theta basis
    Dims dh;                 // one folded half: N_phi / 2 lines per (element, r, theta) row
    int nfold;               // fields the folding buffers hold
    double* Y;               // folded inputs, nfold x P values (double, or float)
    double* Z;               // folded contraction results
    double* Dt2[2];          // dense even / odd extension operators: derivative
    double* Ft2[2];          //   and filter
    double* Dts[2];          // reflection-split copies (nullptr: dense only)
    double* Fts[2];
    uint8_t* fx_dt[2];       // digit-slice images (nullptr: FP64 units)
    uint8_t* fx_ft[2];
    uint8_t* tc_t[2];        // mixed-precision images of the derivative operators
    FoldJob* fjobs;          // fold / unfold job lists (offsets below)
    int fj_first[3], fj_first_u[3], fj_second, fj_second_u, fj_filter[3][2], fj_filter_u[3][2];
    int fj_dbg, fj_dbg_u;
    int job_fy[2];           // FP64 contraction jobs over the folded halves (even, odd)
    int tc_fy[2][2];         // [source FP64 / FP32][even, odd] tensor-core jobs over the halves
    // host copies
    std::vector<double> r_nodes, th_nodes, ph_nodes, rscale_h;
    // instances of the group (concatenated along r)
    int n_inst;
    std::vector<int> inst_E, inst_off;      // elements per instance, first element
    std::vector<double> inst_M, inst_a;     // Kerr-Schild background per instance
    std::vector<int> elem_inst;
    // graph
    cudaGraphExec_t gexec;
    int g_nsteps;
    int g_auto_dt;
    long long launches_per_call;
    long long launches_tmp;
    char err[512];
};

struct grmhd_batch {
    int n;                       // instances
    int ngroups;
    grmhd_ctx** groups;          // one context per group of compatible instances
    std::vector<int> grp, idx;   // instance -> (group, index inside the group)
    cudaStream_t stream;
    bool own_stream;
    cudaGraphExec_t gexec;
    int g_nsteps;
    long long launches_per_step;
    char err[256];
};

static int set_err(grmhd_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return set_err(c, GRMHD_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Sign of each canonical variable under the double-Fourier extension of the Fourier theta
// basis, i.e. under the chart change (theta, phi) -> (-theta, phi + pi) that reaches a point
// across the pole: -1 per theta index of a coordinate-basis component, and -1 once more
// for the sqrt(gamma)-weighted Valencia variables (sqrt(gamma) changes sign with
// sin(theta), so the odd extension is the smooth one).
static const int kThetaParity[NV_MAX] = {
    1, -1, 1, 1, -1, 1,   // gammatilde_{rr, r th, r ph, th th, th ph, ph ph}
    1,                    // conformal factor phi
    1, -1, 1, 1, -1, 1,   // Atilde_ij
    1,                    // K
    1, -1, 1,             // Gammatilde^i
    1,                    // alpha
    1, -1, 1,             // beta^i
    1, -1, 1,             // B^i (Gamma-driver)
    -1,                   // sqrt(gamma) D
    -1, 1, -1,            // sqrt(gamma) S_i
    -1,                   // sqrt(gamma) tau
    -1, 1, -1,            // sqrt(gamma) B^i
    1};                   // psi (GLM)

extern "C" int grmhd_defaults(grmhd_grid* g, grmhd_physics* ph, grmhd_opts* o) {
    if (g) {
        g->n_elem = 2; g->r_min = 1.8; g->r_max = 20.0; g->elem_map = 1;
        g->n_r = 12; g->n_theta = 12; g->n_phi = 16;
        g->theta_min = M_PI / 8; g->theta_max = 7 * M_PI / 8;
        g->theta_basis = 0;
    }
    if (ph) { ph->M = 1.0; ph->a = 0.5; ph->gamma_eos = 4.0 / 3.0; ph->rho_atm = 1e-12; ph->eps_atm = 1e-10; }
    if (o) {
        o->precision = 0; o->integrator = 0; o->evolve_metric = 1; o->gauge = 0;
        o->eta = 2.0; o->cfl = 0.3; o->filter = 47; o->filt_alpha = 36.0; o->filt_p = 8.0;
        o->dealias23_phi = 1; o->c2p_maxit = 60; o->c2p_tol = 1e-15;
        o->contraction = 0;
        o->coupling = 0;
        o->glm = 0; o->glm_ch = 1.0; o->glm_tau = 1.0;
        o->dealias23_theta = 1;
        o->c2p_lambda = 0.0;
    }
    return GRMHD_OK;
}

static int validate(const grmhd_grid* g, const grmhd_physics* ph, const grmhd_opts* o, char* msg) {
    if (!g || !ph || !o) { strcpy(msg, "NULL parameter struct"); return GRMHD_EINVAL; }
    if (g->n_elem < 1 || g->n_elem > 4096) { strcpy(msg, "n_elem out of range"); return GRMHD_EINVAL; }
    if (g->n_r < 4 || g->n_r > 64) { strcpy(msg, "n_r must be in [4, 64]"); return GRMHD_EINVAL; }
    if (g->n_theta < 4 || g->n_theta > 128) { strcpy(msg, "n_theta must be in [4, 128]"); return GRMHD_EINVAL; }
    if (g->n_phi < 4 || g->n_phi > 128 || (g->n_phi % 2)) { strcpy(msg, "n_phi must be even in [4, 128]"); return GRMHD_EINVAL; }
    if (!(g->r_min > 0.0) || !(g->r_max > g->r_min)) { strcpy(msg, "need 0 < r_min < r_max"); return GRMHD_EINVAL; }
    if (!(g->theta_min >= 0.0) || !(g->theta_max > g->theta_min) || !(g->theta_max <= M_PI + 1e-12)) {
        strcpy(msg, "need 0 <= theta_min < theta_max <= pi"); return GRMHD_EINVAL;
    }
    if (g->elem_map != 0 && g->elem_map != 1) { strcpy(msg, "elem_map must be 0 or 1"); return GRMHD_EINVAL; }
    if (g->theta_basis != 0 && g->theta_basis != 1) { strcpy(msg, "theta_basis must be 0 or 1"); return GRMHD_EINVAL; }
    if (g->theta_basis == 1 && (g->theta_min != 0.0 || std::fabs(g->theta_max - M_PI) > 1e-12)) {
        strcpy(msg, "the Fourier theta basis covers the sphere: theta_min = 0, theta_max = pi"); return GRMHD_EINVAL;
    }
    if (!(ph->M > 0.0) || !(std::fabs(ph->a) < ph->M)) { strcpy(msg, "need M > 0 and |a| < M"); return GRMHD_EINVAL; }
    if (!(ph->gamma_eos > 1.0)) { strcpy(msg, "gamma_eos must exceed 1"); return GRMHD_EINVAL; }
    if (!(ph->rho_atm > 0.0) || !(ph->eps_atm >= 0.0)) { strcpy(msg, "bad floors"); return GRMHD_EINVAL; }
    if (o->precision < 0 || o->precision > 2) { strcpy(msg, "precision must be 0, 1 or 2"); return GRMHD_EUNSUPPORTED; }
    if (o->precision > 0 && (g->n_r > 128 || g->n_theta > 128 || g->n_phi > 128)) {
        strcpy(msg, "tensor-core contractions support at most 128 nodes per direction");
        return GRMHD_EUNSUPPORTED;
    }
    if (o->integrator != 0 && o->integrator != 1) { strcpy(msg, "integrator must be 0 or 1"); return GRMHD_EINVAL; }
    if (o->gauge != 0 && o->gauge != 1) { strcpy(msg, "gauge must be 0 or 1"); return GRMHD_EINVAL; }
    if (!(o->cfl > 0.0) || o->c2p_maxit < 1 || !(o->c2p_tol > 0.0)) { strcpy(msg, "bad cfl / c2p options"); return GRMHD_EINVAL; }
    if (o->filter < 0 || o->filter > 63) { strcpy(msg, "filter mask must be in [0, 63]"); return GRMHD_EINVAL; }
    if (o->contraction != 0 && o->contraction != 1) { strcpy(msg, "contraction must be 0 or 1"); return GRMHD_EINVAL; }
    if (o->coupling != 0 && o->coupling != 1) { strcpy(msg, "coupling must be 0 or 1"); return GRMHD_EINVAL; }
    if (o->glm != 0 && o->glm != 1) { strcpy(msg, "glm must be 0 or 1"); return GRMHD_EINVAL; }
    if (o->glm && (!(o->glm_ch >= 0.0) || !(o->glm_tau > 0.0))) { strcpy(msg, "need glm_ch >= 0 and glm_tau > 0"); return GRMHD_EINVAL; }
    if (o->dealias23_theta != 0 && o->dealias23_theta != 1) { strcpy(msg, "dealias23_theta must be 0 or 1"); return GRMHD_EINVAL; }
    if (!(o->c2p_lambda >= 0.0 && o->c2p_lambda <= 1.0)) { strcpy(msg, "c2p_lambda must be in [0, 1]"); return GRMHD_EINVAL; }
    return GRMHD_OK;
}

static void free_ctx(grmhd_ctx* c) {
    if (!c) return;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    double** bufs[] = {&c->U[0], &c->U[1], &c->U[2], &c->acc, &c->prim, &c->flux, &c->tmn, &c->lam,
                       &c->d1, &c->d2, &c->divF, &c->scratch, &c->Dr, &c->Dt, &c->Dp, &c->Fr,
                       &c->Ft, &c->Fp, &c->r_scale, &c->wq, &c->hmin, &c->dt, &c->diag, &c->divB, &c->ham, &c->met};
    for (double** b : bufs)
        if (*b) cudaFree(*b);
    for (int k = 0; k < 3; k++) {
        if (c->Ds[k]) cudaFree(c->Ds[k]);
        if (c->Fs[k]) cudaFree(c->Fs[k]);
    }
    if (c->iface_dev) cudaFree(c->iface_dev);
    if (c->elem_inst_dev) cudaFree(c->elem_inst_dev);
    if (c->nfail) cudaFree(c->nfail);
    if (c->lam_bits) cudaFree(c->lam_bits);
    if (c->nan_flag) cudaFree(c->nan_flag);
    if (c->jobs) cudaFree(c->jobs);
    for (int k = 0; k < 3; k++) {
        if (c->tc_img[k]) cudaFree(c->tc_img[k]);
        if (c->fx_d[k]) cudaFree(c->fx_d[k]);
        if (c->fx_f[k]) cudaFree(c->fx_f[k]);
    }
    if (c->tcjobs) cudaFree(c->tcjobs);
    if (c->tc_err) cudaFree(c->tc_err);
    double** fbufs[] = {&c->Y, &c->Z, &c->Dt2[0], &c->Dt2[1], &c->Ft2[0], &c->Ft2[1], &c->Dts[0], &c->Dts[1],
                        &c->Fts[0], &c->Fts[1]};
    for (double** b : fbufs)
        if (*b) cudaFree(*b);
    for (int k = 0; k < 2; k++) {
        if (c->fx_dt[k]) cudaFree(c->fx_dt[k]);
        if (c->fx_ft[k]) cudaFree(c->fx_ft[k]);
        if (c->tc_t[k]) cudaFree(c->tc_t[k]);
    }
    if (c->fjobs) cudaFree(c->fjobs);
    if (c->s2) cudaStreamDestroy(c->s2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

template <class T>
static cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, n * sizeof(T) + 16);
}

static cudaError_t upload(double* dst, const std::vector<double>& v, cudaStream_t s) {
    return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, s);
}

// Instances that share the node counts, the theta range, the equation of state, the
// floors and the options form one group: they are concatenated along r as radial
// elements of one grid (the right-hand side never uses M or a: the background enters
// only through the initial data), with per-element flags for interface coupling and
// the outer-boundary freeze and per-instance dt.
static bool same_group(const grmhd_grid& g0, const grmhd_physics& p0, const grmhd_grid& g,
                       const grmhd_physics& p) {
    return g.n_r == g0.n_r && g.n_theta == g0.n_theta && g.n_phi == g0.n_phi &&
           g.theta_min == g0.theta_min && g.theta_max == g0.theta_max && g.theta_basis == g0.theta_basis &&
           p.gamma_eos == p0.gamma_eos && p.rho_atm == p0.rho_atm && p.eps_atm == p0.eps_atm;
}

// The contraction tuning table a previous autotuner run stored: the file GRMHD_TUNING_FILE
// names, else fx_tuning.txt next to this library; lines "direction nodes accumulators sets"
// ('#' starts a comment).  Read once per process, at the first context or batch.
static std::once_flag g_tuning_once;
extern "C" int grmhd_create(const grmhd_grid*, const grmhd_physics*, const grmhd_opts*, void*, grmhd_ctx**);
static void load_tuning_file() {
    std::string path;
    const char* env = getenv("GRMHD_TUNING_FILE");
    if (env && *env) {
        path = env;
    } else {
        Dl_info info;
        if (!dladdr((void*)&grmhd_create, &info) || !info.dli_fname) return;
        path = info.dli_fname;
        const size_t pos = path.rfind('/');
        path = (pos == std::string::npos ? std::string() : path.substr(0, pos + 1)) + "fx_tuning.txt";
    }
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return;
    char line[256];
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        int dir, n, kind, ts;
        if (sscanf(line, "%d %d %d %d", &dir, &n, &kind, &ts) == 4 && dir >= 0 && dir <= 2 && n >= 2 && n <= 128 &&
            (kind == 0 || kind == 1) && ts >= 0 && ts <= 2)
            fx_tune_set(dir, n, kind, ts);
    }
    fclose(f);
}

static int ctx_create(int ninst, const grmhd_grid* grids, const grmhd_physics* physs,
                      const grmhd_opts* opts, void* cuda_stream, grmhd_ctx** out) {
    std::call_once(g_tuning_once, load_tuning_file);
    if (!out || ninst < 1 || !grids || !physs || !opts) return GRMHD_EINVAL;
    *out = nullptr;
    char msg[256] = {0};
    for (int i = 0; i < ninst; i++) {
        int st = validate(&grids[i], &physs[i], opts, msg);
        if (st != GRMHD_OK) return st;
        if (!same_group(grids[0], physs[0], grids[i], physs[i])) return GRMHD_EINVAL;
    }
    const grmhd_grid* grid = &grids[0];
    const grmhd_physics* phys = &physs[0];
    // value-initialisation zeroes every plain member and constructs the vectors
    grmhd_ctx* c = new (std::nothrow) grmhd_ctx();
    if (!c) return GRMHD_ENOMEM;
    c->grid = *grid;
    c->phys = *phys;
    c->opts = *opts;
    c->n_inst = ninst;
    int E = 0;
    for (int i = 0; i < ninst; i++) {
        c->inst_off.push_back(E);
        c->inst_E.push_back(grids[i].n_elem);
        c->inst_M.push_back(physs[i].M);
        c->inst_a.push_back(physs[i].a);
        E += grids[i].n_elem;
    }
    const int Nr = grid->n_r, Nt = grid->n_theta, Np = grid->n_phi;
    c->d.E = E; c->d.Nr = Nr; c->d.Nt = Nt; c->d.Np = Np;
    c->d.NtNp = (long long)Nt * Np;
    c->d.elem = c->d.NtNp * Nr;
    c->d.P = c->d.elem * E;
    const long long P = c->d.P;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        // capture needs a non-legacy stream; a blocking stream stays ordered with the
        // legacy default stream the caller named
        cudaError_t e = cudaStreamCreate(&c->stream);
        if (e != cudaSuccess) { free_ctx(c); return GRMHD_ECUDA; }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        free_ctx(c);
        return GRMHD_ECUDA;
    }
    // physics parameters
    c->pp.M = phys->M; c->pp.a = phys->a; c->pp.gam = phys->gamma_eos;
    c->pp.rho_atm = phys->rho_atm; c->pp.eps_atm = phys->eps_atm;
    c->pp.eta = opts->eta; c->pp.gauge = opts->gauge; c->pp.evolve_metric = opts->evolve_metric;
    c->pp.evolve_fluid = 1;
    c->pp.glm = opts->glm;
    c->pp.glm_ch2 = opts->glm_ch * opts->glm_ch;
    c->pp.glm_itau = 1.0 / opts->glm_tau;
    c->nv = NV + opts->glm;
    const int nv = c->nv, glm = opts->glm;
    c->pp.c2p_maxit = opts->c2p_maxit; c->pp.c2p_tol = opts->c2p_tol; c->pp.c2p_lambda = opts->c2p_lambda;
    std::vector<double> wcgl = quad_weights(Nr, true);
    c->pp.w_end = wcgl[0];

    // grid: element bounds of every instance, concatenated
    std::vector<double> xr = cgl_nodes(Nr), xt = gauss_nodes(Nt);
    c->r_nodes.resize((size_t)E * Nr);
    c->rscale_h.resize(E);
    c->elem_inst.resize(E);
    std::vector<unsigned char> iface(E, 0);
    for (int in = 0; in < ninst; in++) {
        const grmhd_grid& gi = grids[in];
        const int Ei = gi.n_elem, off = c->inst_off[in];
        for (int e = 0; e < Ei; e++) {
            double a = gi.elem_map == 1 ? gi.r_min * std::pow(gi.r_max / gi.r_min, (double)e / Ei)
                                        : gi.r_min + (gi.r_max - gi.r_min) * e / Ei;
            double b = gi.elem_map == 1 ? gi.r_min * std::pow(gi.r_max / gi.r_min, (double)(e + 1) / Ei)
                                        : gi.r_min + (gi.r_max - gi.r_min) * (e + 1) / Ei;
            if (e == 0) a = gi.r_min;
            if (e == Ei - 1) b = gi.r_max;
            c->rscale_h[off + e] = 2.0 / (b - a);
            for (int i = 0; i < Nr; i++) c->r_nodes[(size_t)(off + e) * Nr + i] = 0.5 * (a + b) + 0.5 * (b - a) * xr[i];
            c->elem_inst[off + e] = in;
            iface[off + e] = e < Ei - 1;
        }
    }
    double tscale = 2.0 / (grid->theta_max - grid->theta_min);
    c->ft = grid->theta_basis == 1;
    c->th_nodes.resize(Nt);
    for (int k = 0; k < Nt; k++)
        c->th_nodes[k] = c->ft ? (k + 0.5) * M_PI / Nt
                               : grid->theta_min + 0.5 * (grid->theta_max - grid->theta_min) * (1.0 + xt[k]);
    c->ph_nodes.resize(Np);
    for (int l = 0; l < Np; l++) c->ph_nodes[l] = 2.0 * M_PI * l / Np;

    std::vector<double> Dr = cheb_lobatto_D(Nr), Dt = cheb_gauss_D(Nt), Dp = fourier_D_row(Np);
    for (double& v : Dt) v *= tscale;
    std::vector<double> Fr = cheb_filter_matrix(Nr, true, opts->filt_alpha, opts->filt_p);
    std::vector<double> Ft = cheb_filter_matrix(Nt, false, opts->filt_alpha, opts->filt_p);
    std::vector<double> Fp = fourier_filter_row(Np, opts->filt_alpha, opts->filt_p, opts->dealias23_phi != 0);
    // quadrature weights and the CFL spacing
    // theta weights: Fejer weights of the Chebyshev-Gauss nodes, divided by the map's
    // d theta / dx (Chebyshev basis) or, Fourier basis, by sin(theta) (x = -cos(theta)
    // carries the uniform nodes into the Chebyshev-Gauss points; exact for
    // sqrt(gamma)-weighted integrands)
    std::vector<double> wt = quad_weights(Nt, false);
    for (int k = 0; k < Nt; k++) wt[k] = c->ft ? wt[k] / std::sin(c->th_nodes[k]) : wt[k] / tscale;
    std::vector<double> wq((size_t)P);
    std::vector<double> hmin(ninst, 1e300);
    for (int e = 0; e < E; e++)
        for (int i = 0; i < Nr; i++) {
            const double* rn = &c->r_nodes[(size_t)e * Nr];
            double dr = i == 0 ? rn[1] - rn[0] : (i == Nr - 1 ? rn[i] - rn[i - 1] : std::fmin(rn[i] - rn[i - 1], rn[i + 1] - rn[i]));
            for (int k = 0; k < Nt; k++) {
                const double* tn = c->th_nodes.data();
                double dth = k == 0 ? tn[1] - tn[0] : (k == Nt - 1 ? tn[k] - tn[k - 1] : std::fmin(tn[k] - tn[k - 1], tn[k + 1] - tn[k]));
                double r = rn[i];
                double h = std::fmin(std::fmin(dr, r * dth), r * std::sin(tn[k]) * (2.0 * M_PI / Np));
                hmin[c->elem_inst[e]] = std::fmin(hmin[c->elem_inst[e]], h);
                for (int l = 0; l < Np; l++)
                    wq[(((size_t)e * Nr + i) * Nt + k) * Np + l] =
                        wcgl[i] / c->rscale_h[e] * wt[k] * (2.0 * M_PI / Np);
            }
        }

    // device memory
    cudaError_t ce = cudaSuccess;
#define AL(ptr, n) if (ce == cudaSuccess) ce = dalloc(&(ptr), (size_t)(n))
    for (int b = 0; b < 3; b++) AL(c->U[b], nv * P);
    if (opts->integrator == 1) AL(c->acc, nv * P);
    AL(c->prim, N_PRIM * P);
    AL(c->flux, N_FLUX * P);
    AL(c->tmn, N_TMN * P);
    AL(c->lam, P);
    AL(c->d1, (N_D1 + glm) * 3 * P);
    if (glm) AL(c->divB, P);
    AL(c->d2, N_D2 * 6 * P);
    AL(c->divF, 8 * P);
    AL(c->ham, P);
    AL(c->met, 9 * P);
    AL(c->scratch, nv * P);
    AL(c->Dr, Nr * Nr); AL(c->Dt, Nt * Nt); AL(c->Dp, Np);
    AL(c->Fr, Nr * Nr); AL(c->Ft, Nt * Nt); AL(c->Fp, Np);
    AL(c->r_scale, E); AL(c->wq, P); AL(c->hmin, ninst); AL(c->dt, ninst); AL(c->diag, 8);
    AL(c->nfail, 1); AL(c->lam_bits, ninst); AL(c->nan_flag, 1); AL(c->tc_err, 1);
    AL(c->iface_dev, E); AL(c->elem_inst_dev, E);
    // folding buffers of the Fourier theta basis: the first-derivative list (21 fields + 8
    // fluxes, + psi and B^theta with GLM) and, after it, the second-derivative list (22), whose
    // contractions run on the side stream while the flux divergences run on the main one
    c->nfold = N_D1 + 8 + 2 * glm + 2 * N_D2;
    if (c->ft) { AL(c->Y, (long long)c->nfold * P); AL(c->Z, (long long)c->nfold * P); }
#undef AL
    if (ce != cudaSuccess) {
        free_ctx(c);
        return ce == cudaErrorMemoryAllocation ? GRMHD_ENOMEM : GRMHD_ECUDA;
    }
    c->d.iface_next = c->iface_dev;
    c->d.elem_inst = c->elem_inst_dev;
    // job lists
    std::vector<DerivJob> jobs;
    auto add = [&](const double* s, double* dd, int acc) { DerivJob j; j.src = s; j.dst = dd; j.accumulate = acc; j.pad = 0; jobs.push_back(j); };
    for (int b = 0; b < 3; b++)
        for (int dir = 0; dir < 3; dir++) {
            c->job_first[b][dir] = (int)jobs.size();
            for (int f = 0; f < N_D1; f++) add(c->U[b] + (long long)f * P, c->d1 + ((long long)f * 3 + dir) * P, 0);
            if (glm) add(c->U[b] + (long long)V_PSI * P, c->d1 + ((long long)N_D1 * 3 + dir) * P, 0);
            for (int v = 0; v < 8; v++) add(c->flux + ((long long)dir * 8 + v) * P, c->divF + (long long)v * P, dir > 0);
            if (glm) add(c->U[b] + (long long)(V_B + dir) * P, c->divB, dir > 0);
        }
    c->job_first_n = N_D1 + 8 + 2 * glm;
    const int vars2[N_D2] = {0, 1, 2, 3, 4, 5, 6, 17, 18, 19, 20};
    // second derivatives, each mixed pair with the cheaper outer operator (same map: the
    // operators commute, and D_theta commutes with the interface mean):
    //   r:     rr = D_r(mean d_r u), r-theta = D_r(d_theta u), r-phi = D_r(d_phi u)
    //   theta: theta-theta = D_theta(d_theta u), theta-phi = D_theta(d_phi u)
    //   phi:   phi-phi = D_phi(d_phi u)
    // the three radial results are interface-averaged afterwards (pairs rr, rth, rph are
    // the d2 slots 0, 1, 2 of each field)
    c->job_second[0] = (int)jobs.size();
    for (int s = 0; s < N_D2; s++) {
        add(c->d1 + ((long long)vars2[s] * 3 + 0) * P, c->d2 + ((long long)s * 6 + 0) * P, 0);
        add(c->d1 + ((long long)vars2[s] * 3 + 1) * P, c->d2 + ((long long)s * 6 + 1) * P, 0);
        add(c->d1 + ((long long)vars2[s] * 3 + 2) * P, c->d2 + ((long long)s * 6 + 2) * P, 0);
    }
    c->job_second_n[0] = 3 * N_D2;
    c->job_second[1] = (int)jobs.size();
    for (int s = 0; s < N_D2; s++) {
        add(c->d1 + ((long long)vars2[s] * 3 + 1) * P, c->d2 + ((long long)s * 6 + 3) * P, 0);
        add(c->d1 + ((long long)vars2[s] * 3 + 2) * P, c->d2 + ((long long)s * 6 + 4) * P, 0);
    }
    c->job_second_n[1] = 2 * N_D2;
    c->job_second[2] = (int)jobs.size();
    for (int s = 0; s < N_D2; s++)
        add(c->d1 + ((long long)vars2[s] * 3 + 2) * P, c->d2 + ((long long)s * 6 + 5) * P, 0);
    c->job_second_n[2] = N_D2;
    // filter chains: r: U[b] -> scratch; theta: scratch -> U[b]; phi: U[b] -> U[0]
    for (int b = 0; b < 3; b++)
        for (int dir = 0; dir < 3; dir++)
            for (int grp = 0; grp < 2; grp++) {
                c->job_filter[b][dir][grp] = (int)jobs.size();
                const double* src = dir == 0 ? c->U[b] : (dir == 1 ? c->scratch : c->U[b]);
                double* dst = dir == 0 ? c->scratch : (dir == 1 ? c->U[b] : c->U[0]);
                int v0 = grp == 0 ? V_D : 0, ng = grp == 0 ? 8 + glm : N_BSSN;
                for (int v = v0; v < v0 + ng; v++) add(src + (long long)v * P, dst + (long long)v * P, 0);
            }
    c->job_dbg = (int)jobs.size();
    for (int k = 0; k < 64; k++) add(nullptr, nullptr, 0);
    // Fourier theta: contractions of the folded halves, field i at Y / Z + i P (the half
    // for the even operator first, P / 2 values each)
    for (int h = 0; h < 2; h++) {
        c->job_fy[h] = (int)jobs.size();
        if (c->ft)
            for (int i = 0; i < c->nfold; i++)
                add(c->Y + (long long)i * P + h * (P / 2), c->Z + (long long)i * P + h * (P / 2), 0);
    }
    if (dalloc(&c->jobs, jobs.size()) != cudaSuccess) { free_ctx(c); return GRMHD_ENOMEM; }
    cudaStream_t s = c->stream;
    if (cudaMemcpyAsync(c->jobs, jobs.data(), jobs.size() * sizeof(DerivJob), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        upload(c->Dr, Dr, s) != cudaSuccess || upload(c->Dt, Dt, s) != cudaSuccess ||
        upload(c->Dp, Dp, s) != cudaSuccess || upload(c->Fr, Fr, s) != cudaSuccess ||
        upload(c->Ft, Ft, s) != cudaSuccess || upload(c->Fp, Fp, s) != cudaSuccess ||
        upload(c->r_scale, c->rscale_h, s) != cudaSuccess || upload(c->wq, wq, s) != cudaSuccess ||
        upload(c->hmin, hmin, s) != cudaSuccess ||
        cudaMemsetAsync(c->dt, 0, sizeof(double) * ninst, s) != cudaSuccess ||
        cudaMemcpyAsync(c->iface_dev, iface.data(), E, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->elem_inst_dev, c->elem_inst.data(), sizeof(int) * E, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->prim, 0, sizeof(double) * N_PRIM * P, s) != cudaSuccess ||
        cudaMemsetAsync(c->U[0], 0, sizeof(double) * nv * P, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        free_ctx(c);
        return GRMHD_ECUDA;
    }
    // reflection-split copies of the six operators
    {
        const int Ns[3] = {Nr, Nt, Np};
        std::vector<double> dense_d[3] = {Dr, Dt, circulant(Dp)};
        std::vector<double> dense_f[3] = {Fr, Ft, circulant(Fp)};
        for (int k = 0; k < 3; k++) {
            if (!eo_supported(k, Ns[k])) continue;
            std::vector<double> sd = split_operator(dense_d[k], Ns[k], k == 2 ? 1 : 0);
            std::vector<double> sf = split_operator(dense_f[k], Ns[k], k == 2 ? 1 : 0);
            if (dalloc(&c->Ds[k], sd.size()) != cudaSuccess || dalloc(&c->Fs[k], sf.size()) != cudaSuccess ||
                upload(c->Ds[k], sd, s) != cudaSuccess || upload(c->Fs[k], sf, s) != cudaSuccess) {
                free_ctx(c);
                return GRMHD_ENOMEM;
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) { free_ctx(c); return GRMHD_ECUDA; }
    }
    // Fourier theta: even / odd extension operators (dense, reflection-split, digit slices)
    std::vector<double> ext_d[2], ext_f[2];
    if (c->ft) {
        c->dh = c->d;
        c->dh.Np = Np / 2;
        c->dh.NtNp = (long long)Nt * (Np / 2);
        c->dh.elem = c->dh.NtNp * Nr;
        c->dh.P = P / 2;
        // halved: the fold forms the plain sum and difference of each phi pair
        theta_extension_ops(fourier_D_row(2 * Nt), Nt, &ext_d[0], &ext_d[1], 0.5);
        theta_extension_ops(fourier_filter_row(2 * Nt, opts->filt_alpha, opts->filt_p, opts->dealias23_theta != 0), Nt,
                            &ext_f[0], &ext_f[1], 0.5);
        // the digit-slice kernel stages lines with 16-byte bulk copies: the folded halves
        // need an even number of lines per row
        const bool fx_ok = opts->contraction == 0 && fx_supported(1, Nt) && (Np / 2) % 2 == 0;
        int np_ = 0, kp_ = 0, kc_ = 0;
        fx_geometry(Nt, &np_, &kp_, &kc_);
        for (int h = 0; h < 2; h++) {
            if (dalloc(&c->Dt2[h], (size_t)Nt * Nt) != cudaSuccess || dalloc(&c->Ft2[h], (size_t)Nt * Nt) != cudaSuccess ||
                upload(c->Dt2[h], ext_d[h], s) != cudaSuccess || upload(c->Ft2[h], ext_f[h], s) != cudaSuccess) {
                free_ctx(c);
                return GRMHD_ENOMEM;
            }
            if (eo_supported(1, Nt)) {
                std::vector<double> sd = split_operator(ext_d[h], Nt, 0), sf = split_operator(ext_f[h], Nt, 0);
                if (dalloc(&c->Dts[h], sd.size()) != cudaSuccess || dalloc(&c->Fts[h], sf.size()) != cudaSuccess ||
                    upload(c->Dts[h], sd, s) != cudaSuccess || upload(c->Fts[h], sf, s) != cudaSuccess) {
                    free_ctx(c);
                    return GRMHD_ENOMEM;
                }
            }
            if (fx_ok) {
                std::vector<uint8_t> id = fx_operator_image(ext_d[h], Nt, 1.0, np_, kp_, kc_);
                std::vector<uint8_t> iff = fx_operator_image(ext_f[h], Nt, 1.0, np_, kp_, kc_);
                if (cudaMalloc(&c->fx_dt[h], id.size()) != cudaSuccess || cudaMalloc(&c->fx_ft[h], iff.size()) != cudaSuccess ||
                    cudaMemcpyAsync(c->fx_dt[h], id.data(), id.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                    cudaMemcpyAsync(c->fx_ft[h], iff.data(), iff.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    free_ctx(c);
                    return GRMHD_ENOMEM;
                }
            }
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) { free_ctx(c); return GRMHD_ECUDA; }
    }
    if (kernels_init() != cudaSuccess) { free_ctx(c); return GRMHD_ECUDA; }
    if (cudaMemsetAsync(c->tc_err, 0, sizeof(int), s) != cudaSuccess) { free_ctx(c); return GRMHD_ECUDA; }
    // digit-slice images of the FP64 operators (every direction with at most 64 nodes)
    if (opts->contraction == 0) {
        const int Ns[3] = {Nr, Nt, Np};
        std::vector<double> dense_d[3] = {Dr, Dt, circulant(Dp)};
        std::vector<double> dense_f[3] = {Fr, Ft, circulant(Fp)};
        for (int k = 0; k < 3; k++) {
            if (!fx_supported(k, Ns[k]) || (k == 1 && c->ft)) continue;
            int np_, kp_, kc_;
            fx_geometry(Ns[k], &np_, &kp_, &kc_);
            std::vector<uint8_t> img_f = fx_operator_image(dense_f[k], Ns[k], 1.0, np_, kp_, kc_);
            std::vector<uint8_t> img_d;
            if (k == 0) {
                for (int e = 0; e < E; e++) {
                    std::vector<uint8_t> one = fx_operator_image(dense_d[k], Ns[k], c->rscale_h[e], np_, kp_, kc_);
                    c->fx_estride = (long long)one.size();
                    img_d.insert(img_d.end(), one.begin(), one.end());
                }
            } else {
                img_d = fx_operator_image(dense_d[k], Ns[k], 1.0, np_, kp_, kc_);
            }
            if (cudaMalloc(&c->fx_d[k], img_d.size()) != cudaSuccess ||
                cudaMalloc(&c->fx_f[k], img_f.size()) != cudaSuccess ||
                cudaMemcpyAsync(c->fx_d[k], img_d.data(), img_d.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(c->fx_f[k], img_f.data(), img_f.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                free_ctx(c);
                return GRMHD_ENOMEM;
            }
        }
    }
    // tensor-core operator images and job lists (mixed-precision modes)
    std::vector<TcJob> tj;
    auto addt = [&](const void* src, float* dst, int acc) { TcJob j; j.src = src; j.dst = dst; j.accumulate = acc; j.pad = 0; tj.push_back(j); };
    if (opts->precision > 0) {
        const int tf32 = opts->precision == 2;
        const int Ns[3] = {Nr, Nt, Np};
        std::vector<double> dense_d[3] = {Dr, Dt, circulant(Dp)};
        if (c->ft)
            for (int h = 0; h < 2; h++) {
                std::vector<uint8_t> img = tc_operator_image(ext_d[h], Nt, tf32);
                if (cudaMalloc(&c->tc_t[h], img.size()) != cudaSuccess ||
                    cudaMemcpyAsync(c->tc_t[h], img.data(), img.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    free_ctx(c);
                    return GRMHD_ENOMEM;
                }
            }
        for (int k = 0; k < 3; k++) {
            std::vector<uint8_t> img = tc_operator_image(dense_d[k], Ns[k], tf32);
            if (cudaMalloc(&c->tc_img[k], img.size()) != cudaSuccess ||
                cudaMemcpyAsync(c->tc_img[k], img.data(), img.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                free_ctx(c);
                return GRMHD_ENOMEM;
            }
        }
        float* d1f = reinterpret_cast<float*>(c->d1);
        float* d2f = reinterpret_cast<float*>(c->d2);
        float* dFf = reinterpret_cast<float*>(c->divF);
        for (int b = 0; b < 3; b++)
            for (int dir = 0; dir < 3; dir++) {
                c->tc_first[b][dir] = (int)tj.size();
                for (int f = 0; f < N_D1; f++) addt(c->U[b] + (long long)f * P, d1f + ((long long)f * 3 + dir) * P, 0);
                if (opts->glm) addt(c->U[b] + (long long)V_PSI * P, d1f + ((long long)N_D1 * 3 + dir) * P, 0);
                for (int v = 0; v < 8; v++) addt(c->flux + ((long long)dir * 8 + v) * P, dFf + (long long)v * P, dir > 0);
                if (opts->glm) addt(c->U[b] + (long long)(V_B + dir) * P, reinterpret_cast<float*>(c->divB), dir > 0);
            }
        const int vars2[N_D2] = {0, 1, 2, 3, 4, 5, 6, 17, 18, 19, 20};
        c->tc_second[0] = (int)tj.size();
        for (int q = 0; q < N_D2; q++)
            for (int x = 0; x < 3; x++)
                addt(d1f + ((long long)vars2[q] * 3 + x) * P, d2f + ((long long)q * 6 + x) * P, 0);
        c->tc_second[1] = (int)tj.size();
        for (int q = 0; q < N_D2; q++) {
            addt(d1f + ((long long)vars2[q] * 3 + 1) * P, d2f + ((long long)q * 6 + 3) * P, 0);
            addt(d1f + ((long long)vars2[q] * 3 + 2) * P, d2f + ((long long)q * 6 + 4) * P, 0);
        }
        c->tc_second[2] = (int)tj.size();
        for (int q = 0; q < N_D2; q++)
            addt(d1f + ((long long)vars2[q] * 3 + 2) * P, d2f + ((long long)q * 6 + 5) * P, 0);
        // Fourier theta: the folded halves, FP64 (first derivatives) or FP32 (second) inputs,
        // FP32 results
        float* Yf = reinterpret_cast<float*>(c->Y);
        float* Zf = reinterpret_cast<float*>(c->Z);
        for (int src32 = 0; src32 < 2; src32++)
            for (int h = 0; h < 2; h++) {
                c->tc_fy[src32][h] = (int)tj.size();
                if (c->ft)
                    for (int i = 0; i < c->nfold; i++) {
                        const long long o = (long long)i * P + h * (P / 2);
                        addt(src32 ? (const void*)(Yf + o) : (const void*)(c->Y + o), Zf + o, 0);
                    }
            }
        if (cudaMalloc(&c->tcjobs, tj.size() * sizeof(TcJob)) != cudaSuccess ||
            cudaMemcpyAsync(c->tcjobs, tj.data(), tj.size() * sizeof(TcJob), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(c->tc_err, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
            free_ctx(c);
            return GRMHD_ENOMEM;
        }
    }
    // Fourier theta: fold / unfold job lists of every theta contraction of the pipeline
    if (c->ft) {
        std::vector<FoldJob> fj;
        auto addf = [&](const void* src, void* dst, int par, int acc) {
            FoldJob j; j.src = src; j.dst = dst; j.parity = par; j.accumulate = acc; fj.push_back(j);
        };
        const int mixed = opts->precision > 0;
        float* Yf = reinterpret_cast<float*>(c->Y);
        float* Zf = reinterpret_cast<float*>(c->Z);
        // parity of the i-th job of a first-derivative list: 21 fields (+ psi), the theta
        // fluxes of the 8 Valencia variables (one more theta index), sqrt(gamma) B^theta
        std::vector<int> par1;
        for (int f = 0; f < N_D1; f++) par1.push_back(kThetaParity[f]);
        if (glm) par1.push_back(kThetaParity[V_PSI]);
        for (int v = 0; v < 8; v++) par1.push_back(-kThetaParity[V_D + v]);
        if (glm) par1.push_back(kThetaParity[V_B + 1]);
        const int n1 = c->job_first_n;
        for (int b = 0; b < 3; b++) {
            const DerivJob* jl = &jobs[c->job_first[b][1]];
            c->fj_first[b] = (int)fj.size();
            for (int i = 0; i < n1; i++) addf(jl[i].src, c->Y + (long long)i * P, par1[i], 0);
            c->fj_first_u[b] = (int)fj.size();
            for (int i = 0; i < n1; i++) {
                if (mixed) {
                    const TcJob& t = tj[c->tc_first[b][1] + i];
                    addf(Zf + (long long)i * P, t.dst, par1[i], t.accumulate);
                } else {
                    addf(c->Z + (long long)i * P, jl[i].dst, par1[i], jl[i].accumulate);
                }
            }
        }
        // second derivatives: theta-theta = D_theta(d_theta u) (d_theta u has parity -s),
        // theta-phi = D_theta(d_phi u) (parity s); d2 slots 3 and 4 of each field
        const int v2[N_D2] = {0, 1, 2, 3, 4, 5, 6, 17, 18, 19, 20};
        c->fj_second = (int)fj.size();
        for (int q = 0; q < N_D2; q++)
            for (int x = 0; x < 2; x++) {
                const long long i = n1 + 2 * q + x, so = ((long long)v2[q] * 3 + 1 + x) * P;
                const int par = x == 0 ? -kThetaParity[v2[q]] : kThetaParity[v2[q]];
                if (mixed) addf(reinterpret_cast<const float*>(c->d1) + so, Yf + i * P, par, 0);
                else addf(c->d1 + so, c->Y + i * P, par, 0);
            }
        c->fj_second_u = (int)fj.size();
        for (int q = 0; q < N_D2; q++)
            for (int x = 0; x < 2; x++) {
                const long long i = n1 + 2 * q + x, dof = ((long long)q * 6 + 3 + x) * P;
                const int par = x == 0 ? -kThetaParity[v2[q]] : kThetaParity[v2[q]];
                if (mixed) addf(Zf + i * P, reinterpret_cast<float*>(c->d2) + dof, par, 0);
                else addf(c->Z + i * P, c->d2 + dof, par, 0);
            }
        // filter, theta link of the chain scratch -> U[b] (FP64 at every precision)
        for (int b = 0; b < 3; b++)
            for (int grp = 0; grp < 2; grp++) {
                const int v0 = grp == 0 ? V_D : 0, ng = grp == 0 ? 8 + glm : N_BSSN;
                c->fj_filter[b][grp] = (int)fj.size();
                for (int i = 0; i < ng; i++)
                    addf(c->scratch + (long long)(v0 + i) * P, c->Y + (long long)i * P, kThetaParity[v0 + i], 0);
                c->fj_filter_u[b][grp] = (int)fj.size();
                for (int i = 0; i < ng; i++)
                    addf(c->Z + (long long)i * P, c->U[b] + (long long)(v0 + i) * P, kThetaParity[v0 + i], 0);
            }
        // test hook and diagnostics entries, filled per call
        c->fj_dbg = (int)fj.size();
        for (int i = 0; i < c->nfold; i++) addf(nullptr, nullptr, 1, 0);
        c->fj_dbg_u = (int)fj.size();
        for (int i = 0; i < c->nfold; i++) addf(nullptr, nullptr, 1, 0);
        if (cudaMalloc(&c->fjobs, fj.size() * sizeof(FoldJob)) != cudaSuccess ||
            cudaMemcpyAsync(c->fjobs, fj.data(), fj.size() * sizeof(FoldJob), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            free_ctx(c);
            return GRMHD_ENOMEM;
        }
    }
    *out = c;
    return GRMHD_OK;
}

extern "C" int grmhd_create(const grmhd_grid* grid, const grmhd_physics* phys, const grmhd_opts* opts,
                            void* cuda_stream, grmhd_ctx** out) {
    if (!out) return GRMHD_EINVAL;
    *out = nullptr;
    if (!grid || !phys || !opts) return GRMHD_EINVAL;
    const int st = ctx_create(1, grid, phys, opts, cuda_stream, out);
    // TF32 contractions: created, with the warning that the mode misses the mixed bar
    return (st == GRMHD_OK && opts->precision == 2) ? GRMHD_WPRECISION : st;
}

extern "C" int grmhd_destroy(grmhd_ctx* c) {
    if (!c) return GRMHD_EINVAL;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return GRMHD_OK;
}

extern "C" long long grmhd_num_points(const grmhd_ctx* c) { return c ? c->d.P : -1; }

extern "C" int grmhd_num_vars(const grmhd_ctx* c) { return c ? c->nv : -1; }

extern "C" int grmhd_coords(const grmhd_ctx* c, double* r, double* th, double* ph) {
    if (!c) return GRMHD_EINVAL;
    const Dims& d = c->d;
    for (int e = 0; e < d.E; e++)
        for (int i = 0; i < d.Nr; i++)
            for (int k = 0; k < d.Nt; k++)
                for (int l = 0; l < d.Np; l++) {
                    size_t p = (((size_t)e * d.Nr + i) * d.Nt + k) * d.Np + l;
                    if (r) r[p] = c->r_nodes[(size_t)e * d.Nr + i];
                    if (th) th[p] = c->th_nodes[k];
                    if (ph) ph[p] = c->ph_nodes[l];
                }
    return GRMHD_OK;
}

// ------------------------------------------------------------------ pipeline
// One directional contraction of `njobs` FP64 fields: the digit-sliced tensor-core
// kernel when the context built its images (opts.contraction = 0, at most 128 nodes),
// else the reflection-split kernel when the size has a compiled instance, else the dense
// kernel.  filter = 1 uses the modal filter operator (unscaled), 0 the derivative
// (radial: scaled per element).
//
// Accumulators of the digit-slice kernel: with five, the folded one's FP32 additions leave
// an error of about K 2^-53 of sum_j |D_ij| max_j |u_j| per contraction (3.5e-15 / 7.5e-15
// / 1.4e-14 at 24 / 64 / 128 nodes), the worst case of an FP64 dot product.  A derivative
// whose terms cancel (the phi derivative of a flux that is constant in phi up to small
// noise; the second derivatives, which compose two contractions and amplify the first
// one's error by the operator norm, ~N^2 on Chebyshev nodes) carries that error into the
// right-hand side: on the 393,216-node instance the momentum and energy equations landed
// at 1.0-1.5e-11 of their largest value with five accumulators, against 1-3e-12 for the
// FP64 units.  Every derivative therefore takes a sixth accumulator that keeps the
// digit-order sum 6 exact (combine6 in the kernel): operator error 7e-16 of the bound.
// The filter (one contraction of a smooth state, no cancellation) keeps five.  Above 64
// Chebyshev nodes the digit slices' remaining error (the fixed-point rounding of each line
// against its largest value) reaches 1.5e-11 at 96 theta nodes, against 9.5e-12 for the
// FP64 units, which take those derivatives.  force_fx (the test hook): the digit slices
// whenever the image exists.
static cudaError_t contract(grmhd_ctx* c, int dir, int filter, const DerivJob* jobs, int njobs,
                            bool force_fx = false) {
    if (dir == 1 && c->ft) return cudaErrorInvalidValue;   // theta_fourier below
    const int Ns[3] = {c->d.Nr, c->d.Nt, c->d.Np};
    const bool cheb_d = !filter && dir < 2;
    const uint8_t* fx = filter ? c->fx_f[dir] : ((cheb_d && Ns[dir] > 64 && !force_fx) ? nullptr : c->fx_d[dir]);
    if (fx) return launch_contract_fx(dir, c->d, jobs, njobs, fx, (dir == 0 && !filter) ? c->fx_estride : 0,
                                      c->tc_err, c->stream, 0, filter ? 1 : 0);
    const double* split = filter ? c->Fs[dir] : c->Ds[dir];
    const double* rs = filter ? nullptr : c->r_scale;
    if (split) return launch_deriv_eo(dir, c->d, jobs, njobs, split, filter ? 1 : -1, rs, c->stream);
    const double* dense = filter ? (dir == 0 ? c->Fr : (dir == 1 ? c->Ft : c->Fp))
                                 : (dir == 0 ? c->Dr : (dir == 1 ? c->Dt : c->Dp));
    return launch_deriv(dir, c->d, jobs, njobs, dense, rs, c->stream);
}

// Theta contraction of n fields under the Fourier basis: fold the phi pairs, contract
// the two halves along theta with the even and the odd extension operator, unfold into
// the destinations (4 launches).  stage < 0: FP64 values (digit-slice, reflection-split or
// dense kernel); 0 / 1: the mixed-precision tensor-core kernel on FP64 / FP32 inputs.
// i0: folding-buffer field of the list's first job (lists that may run concurrently use
// disjoint fields)
static cudaError_t theta_fourier(grmhd_ctx* c, int filter, int stage, int fold_off, int unfold_off, int n,
                                 int i0 = 0) {
    cudaError_t e = launch_theta_fold(c->d, c->fjobs + fold_off, n, stage == 1, c->stream);
    if (e != cudaSuccess) return e;
    for (int h = 0; h < 2; h++) {
        if (stage >= 0) {
            e = launch_contract_tc(1, stage, c->dh, c->tcjobs + c->tc_fy[stage][h] + i0, n, c->tc_t[h],
                                   c->opts.precision == 2, c->r_scale, c->tc_err, c->stream);
        } else {
            const uint8_t* fx = filter ? c->fx_ft[h] : c->fx_dt[h];
            const double* split = filter ? c->Fts[h] : c->Dts[h];
            const DerivJob* jb = c->jobs + c->job_fy[h] + i0;
            if (fx) e = launch_contract_fx(1, c->dh, jb, n, fx, 0, c->tc_err, c->stream, 0, filter ? 1 : 0);
            else if (split) e = launch_deriv_eo(1, c->dh, jb, n, split, filter ? 1 : -1, nullptr, c->stream);
            else e = launch_deriv(1, c->dh, jb, n, filter ? c->Ft2[h] : c->Dt2[h], nullptr, c->stream);
        }
        if (e != cudaSuccess) return e;
    }
    c->launches_tmp += 3;   // the caller counts the fourth
    return launch_theta_unfold(c->d, c->fjobs + unfold_off, n, stage >= 0, c->stream);
}

// First derivatives from buffer b.  part 0: the BSSN fields (+ psi) and their interface
// means; part 1: the flux divergence (+ the field divergence with GLM), which needs the
// fluxes of k_prep.
static int enqueue_first_derivs(grmhd_ctx* c, int b, int part) {
    const int nB = N_D1 + c->pp.glm, off = part == 0 ? 0 : nB, n = part == 0 ? nB : c->job_first_n - nB;
    const int mixed = c->opts.precision > 0, tf32 = c->opts.precision == 2;
    for (int dir = 0; dir < 3; dir++) {
        if (dir == 1 && c->ft)
            CK(theta_fourier(c, 0, mixed ? 0 : -1, c->fj_first[b] + off, c->fj_first_u[b] + off, n, off));
        else if (mixed)
            CK(launch_contract_tc(dir, 0, c->d, c->tcjobs + c->tc_first[b][dir] + off, n, c->tc_img[dir], tf32,
                                  c->r_scale, c->tc_err, c->stream));
        else
            CK(contract(c, dir, 0, c->jobs + c->job_first[b][dir] + off, n));
        c->launches_tmp++;
    }
    if (part == 0) {
        if (mixed) CK(launch_iface_avg_f(c->d, reinterpret_cast<float*>(c->d1), 3 * c->d.P, nB, c->stream));
        else CK(launch_iface_avg(c->d, c->d1, 3 * c->d.P, nB, c->stream));
        c->launches_tmp++;
    } else if (c->pp.glm) {
        if (mixed) CK(launch_iface_avg_f(c->d, reinterpret_cast<float*>(c->divB), c->d.P, 1, c->stream));
        else CK(launch_iface_avg(c->d, c->divB, c->d.P, 1, c->stream));
        if (c->d.E > 1) c->launches_tmp++;
    }
    return GRMHD_OK;
}

static int enqueue_second_derivs(grmhd_ctx* c) {
    if (c->opts.precision > 0) {
        const int tf32 = c->opts.precision == 2;
        const int n[3] = {3 * N_D2, 2 * N_D2, N_D2};
        for (int dir = 0; dir < 3; dir++) {
            if (dir == 1 && c->ft)
                CK(theta_fourier(c, 0, 1, c->fj_second, c->fj_second_u, n[dir], c->job_first_n));
            else
                CK(launch_contract_tc(dir, 1, c->d, c->tcjobs + c->tc_second[dir], n[dir], c->tc_img[dir], tf32,
                                      c->r_scale, c->tc_err, c->stream));
            c->launches_tmp++;
        }
        for (int x = 0; x < 3; x++)
            CK(launch_iface_avg_f(c->d, reinterpret_cast<float*>(c->d2) + x * c->d.P, 6 * c->d.P, N_D2, c->stream));
        if (c->d.E > 1) c->launches_tmp += 3;
        return GRMHD_OK;
    }
    for (int dir = 0; dir < 3; dir++) {
        if (dir == 1 && c->ft)
            CK(theta_fourier(c, 0, -1, c->fj_second, c->fj_second_u, c->job_second_n[dir], c->job_first_n));
        else CK(contract(c, dir, 0, c->jobs + c->job_second[dir], c->job_second_n[dir]));
        c->launches_tmp++;
    }
    for (int x = 0; x < 3; x++)
        CK(launch_iface_avg(c->d, c->d2 + x * c->d.P, 6 * c->d.P, N_D2, c->stream));
    if (c->d.E > 1) c->launches_tmp += 3;
    return GRMHD_OK;
}

// one RHS evaluation on state buffer b (Us); output per RKCoef; pp selects the halves of
// a split step (evolve_metric / evolve_fluid)
// the calls between construction and destruction enqueue on stream s
struct OnStream {
    grmhd_ctx* c;
    cudaStream_t saved;
    OnStream(grmhd_ctx* c_, cudaStream_t s) : c(c_), saved(c_->stream) { c->stream = s; }
    ~OnStream() { c->stream = saved; }
};

static int enqueue_stage(grmhd_ctx* c, int b, RKCoef co, double* out, const PhysParams& pp) {
    // Two independent chains until the right-hand side: the BSSN derivatives (first
    // derivatives of the metric fields, interface means, second derivatives; they read only
    // the state) on the side stream, the primitive recovery and the flux divergence on the
    // main stream.  They load different units (tensor / integer pipes against the FP64 pipe).
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->s2, c->ev_fork, 0));
    int st;
    {
        OnStream on(c, c->s2);
        st = enqueue_first_derivs(c, b, 0);
        if (!st && pp.evolve_metric) st = enqueue_second_derivs(c);
        if (!st) CK(cudaEventRecord(c->ev_join, c->s2));
    }
    if (st) return st;
    CK(launch_prep(c->d, pp, c->U[b], c->prim, c->flux, c->tmn, c->lam, c->nfail, c->met, c->stream,
                   c->opts.precision > 0));
    c->launches_tmp++;
    st = enqueue_first_derivs(c, b, 1);
    if (st) return st;
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    CK(launch_rhs(c->d, pp, c->U[0], c->U[b], c->prim, c->flux, c->tmn, c->lam, c->met, c->d1, c->d2,
                  c->divF, c->divB, c->opts.precision > 0, c->r_scale, c->dt, co, out, c->acc, c->stream,
                  c->ham_out));
    c->launches_tmp++;
    return GRMHD_OK;
}

// post-step filter from buffer b into U[0]
static int enqueue_filter(grmhd_ctx* c, int b) {
    const long long P = c->d.P;
    const int m = c->opts.filter;
    for (int dir = 0; dir < 3; dir++) {
        const double* src = dir == 0 ? c->U[b] : (dir == 1 ? c->scratch : c->U[b]);
        double* dst = dir == 0 ? c->scratch : (dir == 1 ? c->U[b] : c->U[0]);
        for (int grp = 0; grp < 2; grp++) {
            int bit = (grp == 0 ? 1 : 8) << dir;
            // the Valencia group carries psi (variable 32, right after them) with GLM
            int v0 = grp == 0 ? V_D : 0, ng = grp == 0 ? 8 + c->pp.glm : N_BSSN;
            if (m & bit) {
                if (dir == 1 && c->ft) CK(theta_fourier(c, 1, -1, c->fj_filter[b][grp], c->fj_filter_u[b][grp], ng));
                else CK(contract(c, dir, 1, c->jobs + c->job_filter[b][dir][grp], ng));
                c->launches_tmp++;
            } else if (src != dst) {
                CK(cudaMemcpyAsync(dst + v0 * P, src + v0 * P, sizeof(double) * ng * P, cudaMemcpyDeviceToDevice, c->stream));
            }
        }
    }
    CK(launch_iface_avg(c->d, c->U[0], P, N_BSSN, c->stream));
    c->launches_tmp++;
    if (c->pp.glm) {
        CK(launch_iface_avg(c->d, c->U[0] + (long long)V_PSI * P, P, 1, c->stream));
        if (c->d.E > 1) c->launches_tmp++;
    }
    return GRMHD_OK;
}

static int enqueue_step(grmhd_ctx* c) {
    int st;
    int last;
    // split coupling: the Runge-Kutta stages advance the fluid on the frozen metric
    PhysParams pp = c->pp;
    if (c->opts.coupling == 1) pp.evolve_metric = 0;
    if (c->opts.integrator == 0) {
        RKCoef s1 = {0.0, 1.0, 0.0, 0.0, 0}, s2 = {0.75, 0.25, 0.0, 0.0, 0}, s3 = {1.0 / 3.0, 2.0 / 3.0, 0.0, 0.0, 0};
        if ((st = enqueue_stage(c, 0, s1, c->U[1], pp))) return st;
        if ((st = enqueue_stage(c, 1, s2, c->U[2], pp))) return st;
        if ((st = enqueue_stage(c, 2, s3, c->U[1], pp))) return st;
        last = 1;
    } else {
        RKCoef k1 = {0, 0, 0.5, 1.0 / 6.0, 1}, k2 = {0, 0, 0.5, 1.0 / 3.0, 2}, k3 = {0, 0, 1.0, 1.0 / 3.0, 2},
               k4 = {0, 0, 0.0, 1.0 / 6.0, 3};
        if ((st = enqueue_stage(c, 0, k1, c->U[1], pp))) return st;
        if ((st = enqueue_stage(c, 1, k2, c->U[2], pp))) return st;
        if ((st = enqueue_stage(c, 2, k3, c->U[1], pp))) return st;
        if ((st = enqueue_stage(c, 1, k4, c->U[2], pp))) return st;
        last = 2;
    }
    if (c->opts.coupling == 1 && c->pp.evolve_metric) {
        // then one forward-Euler step of BSSN + gauge with the fluid frozen
        PhysParams pb = c->pp;
        pb.evolve_fluid = 0;
        const RKCoef eu = {0.0, 1.0, 0.0, 0.0, 0};
        const int nb = last == 1 ? 2 : 1;
        if ((st = enqueue_stage(c, last, eu, c->U[nb], pb))) return st;
        last = nb;
    }
    if (c->opts.filter) return enqueue_filter(c, last);
    CK(cudaMemcpyAsync(c->U[0], c->U[last], sizeof(double) * c->nv * c->d.P, cudaMemcpyDeviceToDevice, c->stream));
    return GRMHD_OK;
}

// ------------------------------------------------------------------ public calls
static int copy_in(grmhd_ctx* c, double* dst, const double* src, size_t n, int on_device) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return GRMHD_OK;
}
static int copy_out(grmhd_ctx* c, double* dst, const double* src, size_t n, int on_device) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return GRMHD_OK;
}

extern "C" int grmhd_set_state(grmhd_ctx* c, const double* state, int on_device) {
    if (!c || !state) return GRMHD_EINVAL;
    CK(cudaMemsetAsync(c->prim, 0, sizeof(double) * N_PRIM * c->d.P, c->stream));
    return copy_in(c, c->U[0], state, (size_t)c->nv * c->d.P, on_device);
}

extern "C" int grmhd_get_state(grmhd_ctx* c, double* state, int on_device) {
    if (!c || !state) return GRMHD_EINVAL;
    return copy_out(c, state, c->U[0], (size_t)c->nv * c->d.P, on_device);
}

// Canonical state (GRMHD_NV x P_i, instance-local layout) of instance `in` of the group:
// Kerr-Schild BSSN data of that instance's background, densitized field from A_phi with
// the grid operators, conserved variables from the primitives (instance-local arrays).
// psi != nullptr: the XCTS slice gamma_ij = psi^4 (flat spherical metric), K = 0 instead of
// Kerr-Schild (conformal metric (r^4 sin^2 theta)^(-1/3) diag(1, r^2, r^2 sin^2 theta) with
// det = 1, phi = ln psi + ln(r^4 sin^2 theta) / 12, Gammatilde^i = -d_j gammatilde^ij in closed
// form, lapse psi^-2, shift and driver zero)
static void build_instance_state(const grmhd_ctx* c, int in, const double* rho, const double* p,
                                 const double* vr, const double* vth, const double* vph,
                                 const double* A_phi, std::vector<double>& U, const double* psi = nullptr) {
    const Dims& d = c->d;
    const int Ei = c->inst_E[in], off = c->inst_off[in];
    const long long Pi = (long long)Ei * d.elem;
    U.assign((size_t)c->nv * Pi, 0.0);   // psi (GLM) starts at zero
    double bssn[24];
    // Kerr-Schild BSSN data depends on (r, theta) only
    for (int e = 0; e < Ei && psi; e++)
        for (int i = 0; i < d.Nr; i++)
            for (int k = 0; k < d.Nt; k++) {
                const double r = c->r_nodes[(size_t)(off + e) * d.Nr + i], th = c->th_nodes[k];
                const double st = std::sin(th), w = r * r * r * r * st * st, f = std::pow(w, -1.0 / 3.0);
                for (int l = 0; l < d.Np; l++) {
                    size_t pt = (((size_t)e * d.Nr + i) * d.Nt + k) * d.Np + l;
                    double b[24] = {0.0};
                    b[0] = f;
                    b[3] = f * r * r;
                    b[5] = f * r * r * st * st;
                    b[6] = std::log(psi[pt]) + std::log(w) / 12.0;
                    b[14] = -4.0 / 3.0 * std::cbrt(r) * std::pow(st, 2.0 / 3.0);
                    b[15] = -2.0 / 3.0 * std::pow(r, -2.0 / 3.0) * std::pow(st, -1.0 / 3.0) * std::cos(th);
                    b[17] = 1.0 / (psi[pt] * psi[pt]);
                    for (int v = 0; v < 24; v++) U[(size_t)v * Pi + pt] = b[v];
                }
            }
    for (int e = 0; e < Ei && !psi; e++)
        for (int i = 0; i < d.Nr; i++)
            for (int k = 0; k < d.Nt; k++) {
                ks_bssn_point(c->inst_M[in], c->inst_a[in], c->r_nodes[(size_t)(off + e) * d.Nr + i], c->th_nodes[k], bssn);
                for (int l = 0; l < d.Np; l++) {
                    size_t pt = (((size_t)e * d.Nr + i) * d.Nt + k) * d.Np + l;
                    for (int v = 0; v < 24; v++) U[(size_t)v * Pi + pt] = bssn[v];
                }
            }
    std::vector<double> Dr = cheb_lobatto_D(d.Nr), Dt = cheb_gauss_D(d.Nt);
    double tscale = 2.0 / (c->grid.theta_max - c->grid.theta_min);
    // Fourier theta basis: A_phi (a covariant phi component, parity +1) differentiated on
    // its double-Fourier extension, d_theta A(theta_k, phi_l) = sum_j c[(k - j) mod 2n]
    // A(theta_j, phi_l) + c[(k + j + 1) mod 2n] A(theta_j, phi_l + pi)
    const int n2 = 2 * d.Nt;
    std::vector<double> crow = fourier_D_row(n2);
    if (c->ft) tscale = 1.0;
    for (int e = 0; e < Ei; e++)
        for (int i = 0; i < d.Nr; i++)
            for (int k = 0; k < d.Nt; k++)
                for (int l = 0; l < d.Np; l++) {
                    size_t pt = (((size_t)e * d.Nr + i) * d.Nt + k) * d.Np + l;
                    double dth = 0.0, drr = 0.0;
                    const int lp = (l + d.Np / 2) % d.Np;
                    for (int j = 0; j < d.Nt; j++) {
                        const size_t row = ((size_t)e * d.Nr + i) * d.Nt + j;
                        if (c->ft)
                            dth += crow[((k - j) % n2 + n2) % n2] * A_phi[row * d.Np + l] +
                                   crow[(k + j + 1) % n2] * A_phi[row * d.Np + lp];
                        else
                            dth += Dt[(size_t)k * d.Nt + j] * A_phi[row * d.Np + l];
                    }
                    for (int j = 0; j < d.Nr; j++)
                        drr += Dr[(size_t)i * d.Nr + j] * A_phi[(((size_t)e * d.Nr + j) * d.Nt + k) * d.Np + l];
                    U[(size_t)V_B * Pi + pt] = dth * tscale;
                    U[(size_t)(V_B + 1) * Pi + pt] = -drr * c->rscale_h[off + e];
                    U[(size_t)(V_B + 2) * Pi + pt] = 0.0;
                }
    for (long long pt = 0; pt < Pi; pt++) {
        double b[24];
        for (int v = 0; v < 24; v++) b[v] = U[(size_t)v * Pi + pt];
        double g[3][3], sqg;
        metric_from_bssn_point(b, g, &sqg);
        double B_u[3] = {U[(size_t)V_B * Pi + pt] / sqg, U[(size_t)(V_B + 1) * Pi + pt] / sqg, U[(size_t)(V_B + 2) * Pi + pt] / sqg};
        double v_u[3] = {vr[pt], vth[pt], vph[pt]};
        double D, S[3], tau;
        prim_to_cons_point(rho[pt], p[pt], v_u, B_u, g, c->phys.gamma_eos, &D, S, &tau);
        U[(size_t)V_D * Pi + pt] = sqg * D;
        for (int j = 0; j < 3; j++) U[(size_t)(V_S + j) * Pi + pt] = sqg * S[j];
        U[(size_t)V_TAU * Pi + pt] = sqg * tau;
    }
}

// copy an instance-local canonical array into / out of the group's state (row v of the
// instance is a contiguous block at element offset inst_off in row v of the group)
static int inst_copy(grmhd_ctx* c, int in, double* dev_rows, long long rows, const double* src, double* dst,
                     int on_device, int to_device) {
    const long long Pi = (long long)c->inst_E[in] * c->d.elem;
    const size_t w = (size_t)Pi * sizeof(double), gp = (size_t)c->d.P * sizeof(double);
    double* base = dev_rows + (long long)c->inst_off[in] * c->d.elem;
    cudaMemcpyKind k = to_device ? (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                                 : (on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    if (to_device) CK(cudaMemcpy2DAsync(base, gp, src, w, w, (size_t)rows, k, c->stream));
    else CK(cudaMemcpy2DAsync(dst, w, base, gp, w, (size_t)rows, k, c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return GRMHD_OK;
}

static int inst_set_state(grmhd_ctx* c, int in, const double* state, int on_device) {
    const long long Pi = (long long)c->inst_E[in] * c->d.elem;
    // reset this instance's primitive guess (the next recovery starts from a bracket)
    CK(cudaMemset2DAsync(c->prim + (long long)c->inst_off[in] * c->d.elem, (size_t)c->d.P * sizeof(double), 0,
                         (size_t)Pi * sizeof(double), N_PRIM, c->stream));
    return inst_copy(c, in, c->U[0], c->nv, state, nullptr, on_device, 1);
}

extern "C" int grmhd_init_prims(grmhd_ctx* c, const double* rho, const double* p, const double* vr,
                                const double* vth, const double* vph, const double* A_phi) {
    NvtxRange nvtx_range("grmhd_init_prims");
    if (!c || !rho || !p || !vr || !vth || !vph || !A_phi) return GRMHD_EINVAL;
    std::vector<double> U;
    for (int in = 0; in < c->n_inst; in++) {
        const long long o = (long long)c->inst_off[in] * c->d.elem;
        build_instance_state(c, in, rho + o, p + o, vr + o, vth + o, vph + o, A_phi + o, U);
        int st = inst_set_state(c, in, U.data(), 0);
        if (st) return st;
    }
    return GRMHD_OK;
}

extern "C" int grmhd_xcts_init(grmhd_ctx* c, const double* rho, const double* p, const double* vr,
                               const double* vth, const double* vph, const double* A_phi, int iters,
                               double tol, double* psi_out, double* changes, double* stats) {
    NvtxRange nvtx_range("grmhd_xcts_init");
    if (!c || !rho || !p || !vr || !vth || !vph || !A_phi || iters < 1 || iters > 10000 || !(tol >= 0.0))
        return GRMHD_EINVAL;
    if (!c->ft) return set_err(c, GRMHD_EUNSUPPORTED, "the XCTS solve covers the whole sphere: theta_basis = 1 only");
    if (c->n_inst != 1) return set_err(c, GRMHD_EUNSUPPORTED, "XCTS initial data is built for one instance");
    const Dims& d = c->d;
    XctsOps o;
    o.E = d.E; o.Nr = d.Nr; o.Nt = d.Nt; o.Np = d.Np;
    const size_t nr2 = (size_t)d.Nr * d.Nr, nt2 = (size_t)d.Nt * d.Nt;
    const std::vector<double> D = cheb_lobatto_D(d.Nr);
    o.Dr.assign(nr2 * d.E, 0.0);
    o.Drr.assign(nr2 * d.E, 0.0);
    for (int e = 0; e < d.E; e++) {
        double* Dr = &o.Dr[nr2 * e];
        for (size_t q = 0; q < nr2; q++) Dr[q] = D[q] * c->rscale_h[e];
        for (int i = 0; i < d.Nr; i++)
            for (int j = 0; j < d.Nr; j++) {
                double acc = 0.0;
                for (int q = 0; q < d.Nr; q++) acc += Dr[(size_t)i * d.Nr + q] * Dr[(size_t)q * d.Nr + j];
                o.Drr[nr2 * e + (size_t)i * d.Nr + j] = acc;
            }
    }
    // theta: the mode's extension parity s = (-1)^m; d_theta of parity s, then of parity -s
    std::vector<double> ev, od;
    theta_extension_ops(fourier_D_row(2 * d.Nt), d.Nt, &ev, &od);
    o.D1.resize(2 * nt2);
    o.D2.assign(2 * nt2, 0.0);
    for (size_t q = 0; q < nt2; q++) { o.D1[q] = ev[q]; o.D1[nt2 + q] = od[q]; }
    for (int i = 0; i < d.Nt; i++)
        for (int j = 0; j < d.Nt; j++) {
            double a = 0.0, b = 0.0;
            for (int q = 0; q < d.Nt; q++) {
                a += od[(size_t)i * d.Nt + q] * ev[(size_t)q * d.Nt + j];
                b += ev[(size_t)i * d.Nt + q] * od[(size_t)q * d.Nt + j];
            }
            o.D2[(size_t)i * d.Nt + j] = a;
            o.D2[nt2 + (size_t)i * d.Nt + j] = b;
        }
    o.r = c->r_nodes;
    o.th = c->th_nodes;
    o.M = c->inst_M[0];
    o.r_min = c->grid.r_min;
    o.r_max = c->grid.r_max;
    // fixed point from the puncture psi = 1 + M / (2 r)
    std::vector<double> psi((size_t)d.P);
    for (int e = 0; e < d.E; e++)
        for (int i = 0; i < d.Nr; i++)
            for (long long kl = 0; kl < d.NtNp; kl++)
                psi[((size_t)e * d.Nr + i) * d.NtNp + kl] = 1.0 + o.M / (2.0 * c->r_nodes[(size_t)e * d.Nr + i]);
    char msg[256] = {0};
    int st = xcts_solve(o, rho, psi.data(), iters, tol, changes, stats, c->stream, msg, sizeof(msg));
    if (st) return set_err(c, st, "%s", msg);
    std::vector<double> U;
    build_instance_state(c, 0, rho, p, vr, vth, vph, A_phi, U, psi.data());
    st = inst_set_state(c, 0, U.data(), 0);
    if (st) return st;
    if (psi_out) memcpy(psi_out, psi.data(), sizeof(double) * (size_t)d.P);
    return GRMHD_OK;
}

extern "C" int grmhd_rhs(grmhd_ctx* c, double* out, int on_device) {
    NvtxRange nvtx_range("grmhd_rhs");
    if (!c || !out) return GRMHD_EINVAL;
    c->launches_tmp = 0;
    CK(cudaMemsetAsync(c->nfail, 0, sizeof(unsigned long long), c->stream));
    RKCoef co = {0, 0, 0, 0, -1};
    double* dst = on_device ? out : c->scratch;
    int st = enqueue_stage(c, 0, co, dst, c->pp);
    if (st) return st;
    c->launches_per_call = c->launches_tmp;
    if (!on_device) return copy_out(c, out, c->scratch, (size_t)c->nv * c->d.P, 0);
    return GRMHD_OK;
}

extern "C" int grmhd_con2prim(grmhd_ctx* c, double* prim_out, int on_device, long long* n_failed) {
    NvtxRange nvtx_range("grmhd_con2prim");
    if (!c) return GRMHD_EINVAL;
    CK(cudaMemsetAsync(c->nfail, 0, sizeof(unsigned long long), c->stream));
    CK(launch_prep(c->d, c->pp, c->U[0], c->prim, c->flux, c->tmn, c->lam, c->nfail, c->met, c->stream));
    if (prim_out) {
        int st = copy_out(c, prim_out, c->prim, (size_t)N_PRIM * c->d.P, on_device);
        if (st) return st;
    }
    if (n_failed) {
        unsigned long long nf = 0;
        CK(cudaMemcpyAsync(&nf, c->nfail, sizeof(nf), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        *n_failed = (long long)nf;
    }
    return GRMHD_OK;
}

extern "C" int grmhd_cfl_dt(grmhd_ctx* c, double* dt) {
    if (!c || !dt) return GRMHD_EINVAL;
    CK(launch_cfl(c->d, c->n_inst, c->U[0], c->hmin, c->opts.cfl, c->dt, c->lam_bits, c->stream));
    CK(cudaMemcpyAsync(dt, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return GRMHD_OK;
}

static int build_graph(grmhd_ctx* c, int nsteps, int auto_dt) {
    NvtxRange nvtx_range("grmhd graph capture");
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int st = GRMHD_OK;
    c->launches_tmp = 0;
    if (auto_dt) {
        cudaError_t e = launch_cfl(c->d, c->n_inst, c->U[0], c->hmin, c->opts.cfl, c->dt, c->lam_bits, c->stream);
        if (e != cudaSuccess) st = set_err(c, GRMHD_ECUDA, "cfl: %s", cudaGetErrorString(e));
        c->launches_tmp += 2;
    }
    for (int s = 0; s < nsteps && st == GRMHD_OK; s++) st = enqueue_step(c);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != GRMHD_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return set_err(c, GRMHD_ECUDA, "capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_err(c, GRMHD_ECUDA, "instantiate: %s", cudaGetErrorString(e));
    c->g_nsteps = nsteps;
    c->g_auto_dt = auto_dt;
    c->launches_per_call = c->launches_tmp;
    return GRMHD_OK;
}

extern "C" int grmhd_step(grmhd_ctx* c, double dt, int nsteps, double* dt_used) {
    NvtxRange nvtx_range("grmhd_step");
    if (!c || nsteps < 1) return GRMHD_EINVAL;
    int auto_dt = !(dt > 0.0);
    if (!c->gexec || c->g_nsteps != nsteps || c->g_auto_dt != auto_dt) {
        int st = build_graph(c, nsteps, auto_dt);
        if (st) return st;
    }
    std::vector<double> dts(c->n_inst, dt);
    if (!auto_dt) CK(cudaMemcpyAsync(c->dt, dts.data(), sizeof(double) * c->n_inst, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->nfail, 0, sizeof(unsigned long long), c->stream));
    CK(cudaGraphLaunch(c->gexec, c->stream));
    CK(cudaMemsetAsync(c->nan_flag, 0, sizeof(int), c->stream));
    CK(launch_nan_check((long long)c->nv * c->d.P, c->U[0], c->nan_flag, c->stream));
    int flag = 0;
    double dtv = dt;
    CK(cudaMemcpyAsync(&flag, c->nan_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&dtv, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (dt_used) *dt_used = dtv;
    if (c->tc_err) {
        int te = 0;
        CK(cudaMemcpy(&te, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (te) {
            CK(cudaMemset(c->tc_err, 0, sizeof(int)));
            return set_err(c, GRMHD_ETIMEOUT, "a tensor-core contraction wait timed out");
        }
    }
    if (flag) return set_err(c, GRMHD_ENAN, "non-finite value in the evolved state");
    return GRMHD_OK;
}

extern "C" int grmhd_diag(grmhd_ctx* c, double out[GRMHD_NDIAG]) {
    NvtxRange nvtx_range("grmhd_diag");
    if (!c || !out) return GRMHD_EINVAL;
    // Hamiltonian constraint: one right-hand-side evaluation of the current state with the
    // metric part always on (its result, written to scratch, is discarded); k_rhs writes H
    // per node from the Ricci tensor it forms anyway
    {
        PhysParams ph = c->pp;
        ph.evolve_metric = 1;
        ph.evolve_fluid = 1;
        const RKCoef co = {0, 0, 0, 0, -1};
        c->ham_out = c->ham;
        const long long keep = c->launches_tmp;
        const int st = enqueue_stage(c, 0, co, c->scratch, ph);
        c->ham_out = nullptr;
        c->launches_tmp = keep;
        if (st) return st;
    }
    CK(cudaMemsetAsync(c->nfail, 0, sizeof(unsigned long long), c->stream));
    CK(launch_prep(c->d, c->pp, c->U[0], c->prim, c->flux, c->tmn, c->lam, c->nfail, c->met, c->stream));
    // divergence of the densitized field into scratch
    const long long P = c->d.P;
    DerivJob jb[3];
    for (int dir = 0; dir < 3; dir++) { jb[dir].src = c->U[0] + (V_B + dir) * P; jb[dir].dst = c->scratch; jb[dir].accumulate = dir > 0; jb[dir].pad = 0; }
    CK(cudaMemcpyAsync(c->jobs + c->job_dbg, jb, sizeof(jb), cudaMemcpyHostToDevice, c->stream));
    for (int dir = 0; dir < 3; dir++) {
        if (dir == 1 && c->ft) {
            // Fourier theta: sqrt(gamma) B^theta through the fold, added into scratch
            FoldJob fj[2];
            fj[0].src = jb[1].src; fj[0].dst = c->Y; fj[0].parity = kThetaParity[V_B + 1]; fj[0].accumulate = 0;
            fj[1].src = c->Z; fj[1].dst = c->scratch; fj[1].parity = kThetaParity[V_B + 1]; fj[1].accumulate = 1;
            CK(cudaMemcpyAsync(c->fjobs + c->fj_dbg, &fj[0], sizeof(FoldJob), cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->fjobs + c->fj_dbg_u, &fj[1], sizeof(FoldJob), cudaMemcpyHostToDevice, c->stream));
            CK(theta_fourier(c, 0, -1, c->fj_dbg, c->fj_dbg_u, 1));
        } else {
            CK(contract(c, dir, 0, c->jobs + c->job_dbg + dir, 1));
        }
    }
    CK(cudaMemsetAsync(c->diag, 0, sizeof(double) * 8, c->stream));
    CK(launch_diag(c->d, c->pp, c->U[0], c->prim, c->wq, c->scratch, c->diag, c->stream, c->ham));
    double h[8];
    unsigned long long nf = 0;
    double dtv = 0.0;
    CK(cudaMemcpyAsync(h, c->diag, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&nf, c->nfail, sizeof(nf), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&dtv, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < GRMHD_NDIAG; i++) out[i] = 0.0;
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = (double)nf;
    out[4] = dtv;
    out[5] = h[5];                                    // max |H|
    out[6] = h[7] > 0.0 ? std::sqrt(h[6] / h[7]) : 0.0;  // quadrature RMS of H
    return GRMHD_OK;
}

extern "C" long long grmhd_launch_count(const grmhd_ctx* c) { return c ? c->launches_per_call : -1; }

// Algorithmic FP64 flops of one contraction of one field over the whole grid: dense
// rows 2 N per output; reflection split per line 2 np (s, a) + np (4 np + 2 nf + 5)
// (pair outputs) + nf (2 np + 2 nf + 1) (fixed-point outputs), np pairs, nf fixed points.
static double contraction_flops(const grmhd_ctx* c, int dir, int filter) {
    const int Ns[3] = {c->d.Nr, c->d.Nt, c->d.Np};
    const int N = Ns[dir];
    const double P = (double)c->d.P;
    const double* split = (dir == 1 && c->ft) ? (filter ? c->Fts[0] : c->Dts[0]) : (filter ? c->Fs[dir] : c->Ds[dir]);
    if (!split) return 2.0 * N * P;
    double np = dir == 2 ? N / 2 - 1 : N / 2, nf = dir == 2 ? 2 : N % 2;
    double per_line = 2 * np + np * (4 * np + 2 * nf + 5) + nf * (2 * np + 2 * nf + 1);
    return per_line * P / N;
}

// Tensor-core contraction of one field: 128-line tiles x (Np x Kp) x slice products x 2.
static double tc_flops(const grmhd_ctx* c, int dir) {
    const int Ns[3] = {c->d.Nr, c->d.Nt, c->d.Np};
    const int N = Ns[dir];
    const double K = (N + 15) / 16 * 16;
    const double lines = dir == 0 ? (double)c->d.E * c->d.NtNp : (dir == 1 ? (double)c->d.E * c->d.Nr * c->d.Np : (double)c->d.P / N);
    const double tiles = std::ceil(lines / 128.0);
    return tiles * 128.0 * K * K * 2.0 * (c->opts.precision == 2 ? 1 : 6);
}

extern "C" int grmhd_kernel_times(grmhd_ctx* c, int reps, double* ms_out, double* flops_out,
                                  double* bytes_out, int n) {
    NvtxRange nvtx_range("grmhd_kernel_times");
    if (!c || !ms_out || reps < 1 || n < 1 || n > GRMHD_NKT) return GRMHD_EINVAL;
    const long long P = c->d.P;
    const int mixed = c->opts.precision > 0, tf32 = c->opts.precision == 2;
    double ms[GRMHD_NKT] = {0}, fl[GRMHD_NKT] = {0}, by[GRMHD_NKT] = {0};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // keep the state: U[1] <- U[0], work on U[1], U[2] holds the saved copy
    CK(cudaMemcpyAsync(c->U[2], c->U[0], sizeof(double) * c->nv * P, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->U[1], c->U[0], sizeof(double) * c->nv * P, cudaMemcpyDeviceToDevice, c->stream));
    RKCoef co = {0, 0, 0, 0, -1};
    int st = GRMHD_OK;
    for (int k = 0; k < GRMHD_NKT && st == GRMHD_OK; k++) {
        // bring the buffers the kernel reads up to date (untimed)
        if (k >= 1) { c->launches_tmp = 0; st = enqueue_stage(c, 1, co, c->scratch, c->pp); if (st) break; }
        CK(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < reps; r++) {
            cudaError_t e = cudaSuccess;
            if (k == 0) e = launch_prep(c->d, c->pp, c->U[1], c->prim, c->flux, c->tmn, c->lam, c->nfail, c->met, c->stream,
                                        mixed);
            else if (k >= 1 && k <= 3) {
                int dir = k - 1;
                if (dir == 1 && c->ft) {
                    e = theta_fourier(c, 0, mixed ? 0 : -1, c->fj_first[1], c->fj_first_u[1], c->job_first_n);
                    fl[k] = mixed ? tc_flops(c, dir) * c->job_first_n : contraction_flops(c, dir, 0) * c->job_first_n;
                    by[k] = (double)P * c->job_first_n * (mixed ? 8.0 + 4.0 : 16.0) + 8.0 * 8.0 * P;
                } else if (mixed) {
                    e = launch_contract_tc(dir, 0, c->d, c->tcjobs + c->tc_first[1][dir], c->job_first_n, c->tc_img[dir], tf32,
                                           c->r_scale, c->tc_err, c->stream);
                    fl[k] = tc_flops(c, dir) * c->job_first_n;
                    by[k] = (double)P * c->job_first_n * (8.0 + 4.0) + (dir > 0 ? (8.0 + c->pp.glm) * 4.0 * P : 0.0);
                } else {
                    e = contract(c, dir, 0, c->jobs + c->job_first[1][dir], c->job_first_n);
                    fl[k] = contraction_flops(c, dir, 0) * c->job_first_n;
                    by[k] = (double)P * c->job_first_n * 16.0 + (dir > 0 ? 8.0 * 8.0 * P : 0.0);
                }
            } else if (k == 4) {
                e = mixed ? launch_iface_avg_f(c->d, reinterpret_cast<float*>(c->d1), 3 * P, N_D1 + c->pp.glm, c->stream)
                          : launch_iface_avg(c->d, c->d1, 3 * P, N_D1 + c->pp.glm, c->stream);
            } else if (k >= 5 && k <= 7) {
                int dir = k - 5;
                const int nj[3] = {3 * N_D2, 2 * N_D2, N_D2};
                if (dir == 1 && c->ft) {
                    e = theta_fourier(c, 0, mixed ? 1 : -1, c->fj_second, c->fj_second_u, nj[dir], c->job_first_n);
                    fl[k] = (mixed ? tc_flops(c, dir) : contraction_flops(c, dir, 0)) * nj[dir];
                    by[k] = (double)P * nj[dir] * (mixed ? 8.0 : 16.0);
                } else if (mixed) {
                    e = launch_contract_tc(dir, 1, c->d, c->tcjobs + c->tc_second[dir], nj[dir], c->tc_img[dir], tf32,
                                           c->r_scale, c->tc_err, c->stream);
                    fl[k] = tc_flops(c, dir) * nj[dir];
                    by[k] = (double)P * nj[dir] * 8.0;
                } else {
                    e = contract(c, dir, 0, c->jobs + c->job_second[dir], c->job_second_n[dir]);
                    fl[k] = contraction_flops(c, dir, 0) * c->job_second_n[dir];
                    by[k] = (double)P * c->job_second_n[dir] * 16.0;
                }
            } else if (k == 8) {
                for (int x = 0; x < 3 && e == cudaSuccess; x++)
                    e = mixed ? launch_iface_avg_f(c->d, reinterpret_cast<float*>(c->d2) + x * P, 6 * P, N_D2, c->stream)
                              : launch_iface_avg(c->d, c->d2 + x * P, 6 * P, N_D2, c->stream);
            }
            else if (k == 9) e = launch_rhs(c->d, c->pp, c->U[0], c->U[1], c->prim, c->flux, c->tmn, c->lam, c->met, c->d1, c->d2,
                                            c->divF, c->divB, c->opts.precision > 0, c->r_scale, c->dt, co, c->scratch,
                                            c->acc, c->stream);
            else {
                int dir = k - 10;
                // filter contraction of all 32 variables of U[1] (scratch <-> U[1] chain)
                if (dir == 1 && c->ft) {
                    e = theta_fourier(c, 1, -1, c->fj_filter[1][1], c->fj_filter_u[1][1], N_BSSN);
                    if (e == cudaSuccess)
                        e = theta_fourier(c, 1, -1, c->fj_filter[1][0], c->fj_filter_u[1][0], 8 + c->pp.glm);
                } else {
                    e = contract(c, dir, 1, c->jobs + c->job_filter[1][dir][1], N_BSSN);
                    if (e == cudaSuccess) e = contract(c, dir, 1, c->jobs + c->job_filter[1][dir][0], 8 + c->pp.glm);
                }
                fl[k] = contraction_flops(c, dir, 1) * c->nv;
                by[k] = (double)P * c->nv * 16.0;
            }
            if (e != cudaSuccess) { st = set_err(c, GRMHD_ECUDA, "kernel_times: %s", cudaGetErrorString(e)); break; }
        }
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        ms[k] = t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaMemcpyAsync(c->U[0], c->U[2], sizeof(double) * c->nv * P, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st) return st;
    for (int k = 0; k < n; k++) {
        ms_out[k] = ms[k];
        if (flops_out) flops_out[k] = fl[k];
        if (bytes_out) bytes_out[k] = by[k];
    }
    return GRMHD_OK;
}

// ------------------------------------------------------------------ contraction autotuner
// The digit-slice contraction can run with one TMEM accumulator set (two CTAs per SM for up
// to 6 x 32 columns) or two (one CTA per SM; the MMAs of the next item overlap the epilogue
// of the previous one).  Which is faster depends on the class (direction, nodes,
// accumulators); the autotuner times both on the context's own buffers and records the
// faster one in the process-wide table every later launch of that class reads.
extern "C" int grmhd_tune_set(int dir, int n, int kind, int tsets) {
    if (dir < 0 || dir > 2 || n < 2 || n > 128 || (kind != 0 && kind != 1) || tsets < 0 || tsets > 2)
        return GRMHD_EINVAL;
    fx_tune_set(dir, n, kind, tsets);
    return GRMHD_OK;
}

extern "C" int grmhd_tune_get(int dir, int n, int kind) {
    if (dir < 0 || dir > 2 || n < 2 || n > 128 || (kind != 0 && kind != 1)) return GRMHD_EINVAL;
    return fx_tune_get(dir, n, kind);
}

extern "C" int grmhd_tune_contractions(grmhd_ctx* c, int nfields, int reps, double* ms_out, int* choice_out) {
    NvtxRange nvtx_range("grmhd_tune_contractions");
    if (!c || nfields < 1 || nfields > 32 || reps < 1) return GRMHD_EINVAL;
    if (c->n_inst != 1) return set_err(c, GRMHD_EUNSUPPORTED, "tuning runs on a single-instance context");
    const long long P = c->d.P;
    std::vector<DerivJob> jb(nfields);
    for (int f = 0; f < nfields; f++) {
        jb[f].src = c->U[0] + (long long)f * P;
        jb[f].dst = c->scratch + (long long)f * P;
        jb[f].accumulate = 0;
        jb[f].pad = 0;
    }
    CK(cudaMemcpyAsync(c->jobs + c->job_dbg, jb.data(), sizeof(DerivJob) * nfields, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return set_err(c, GRMHD_ECUDA, "events"); }
    const int Ns[3] = {c->d.Nr, c->d.Nt, c->d.Np};
    int st = GRMHD_OK;
    for (int dir = 0; dir < 3 && st == GRMHD_OK; dir++)
        for (int kind = 0; kind < 2 && st == GRMHD_OK; kind++) {      // 0 derivative, 1 filter
            const int N = Ns[dir];
            const bool ftd = dir == 1 && c->ft;
            const uint8_t* img = ftd ? (kind == 0 ? c->fx_dt[0] : c->fx_ft[0]) : (kind == 0 ? c->fx_d[dir] : c->fx_f[dir]);
            // Chebyshev derivatives above 64 nodes run on the FP64 units
            if (kind == 0 && dir < 2 && !c->ft && N > 64) img = nullptr;
            const Dims& dd = ftd ? c->dh : c->d;
            const long long estride = (dir == 0 && kind == 0) ? c->fx_estride : 0;
            double best_ms = 1e30;
            int best = 1;
            for (int ts = 1; ts <= 2; ts++) {
                double ms = -1.0;
                if (img && fx_supported(dir, N) && (ts == 1 || fx_two_sets_possible(dir, N))) {
                    cudaError_t e = launch_contract_fx(dir, dd, c->jobs + c->job_dbg, nfields, img, estride, c->tc_err,
                                                       c->stream, 0, kind, ts);
                    cudaEventRecord(e0, c->stream);
                    for (int r = 0; r < reps && e == cudaSuccess; r++)
                        e = launch_contract_fx(dir, dd, c->jobs + c->job_dbg, nfields, img, estride, c->tc_err, c->stream,
                                               0, kind, ts);
                    cudaEventRecord(e1, c->stream);
                    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                        st = set_err(c, GRMHD_ECUDA, "tuning launch: %s", cudaGetErrorString(e));
                        break;
                    }
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = t / reps;
                    // a second set must win by 2 % (launch-to-launch noise is about 1 %)
                    if (ts == 1 || ms < 0.98 * best_ms) { best_ms = ms; best = ts; }
                }
                if (ms_out) ms_out[(dir * 2 + kind) * 2 + (ts - 1)] = ms;
            }
            if (st) break;
            if (img) fx_tune_set(dir, N, kind, best);
            if (choice_out) choice_out[dir * 2 + kind] = img ? best : 0;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    int te = 0;
    CK(cudaMemcpyAsync(&te, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (te) return set_err(c, GRMHD_ETIMEOUT, "a tuning launch timed out");
    return GRMHD_OK;
}

extern "C" int grmhd_debug_deriv(grmhd_ctx* c, const double* in, double* out, int nfields, int dir) {
    if (!c || !in || !out || nfields < 1 || nfields > 64 || dir < 0 || dir > 2) return GRMHD_EINVAL;
    const long long P = c->d.P;
    std::vector<DerivJob> jb(nfields);
    for (int f = 0; f < nfields; f++) { jb[f].src = in + f * P; jb[f].dst = out + f * P; jb[f].accumulate = 0; jb[f].pad = 0; }
    if (dir == 1 && c->ft) {
        std::vector<int> par(nfields, 1);
        return grmhd_debug_theta(c, in, out, nfields, par.data(), 0);
    }
    CK(cudaMemcpyAsync(c->jobs + c->job_dbg, jb.data(), sizeof(DerivJob) * nfields, cudaMemcpyHostToDevice, c->stream));
    CK(contract(c, dir, 0, c->jobs + c->job_dbg, nfields, true));
    CK(cudaStreamSynchronize(c->stream));
    return GRMHD_OK;
}

extern "C" int grmhd_debug_wait_timeout(grmhd_ctx* c) {
    if (!c) return GRMHD_EINVAL;
    int dir = -1;
    for (int k = 0; k < 3 && dir < 0; k++)
        if (c->fx_d[k]) dir = k;
    if (dir < 0) return set_err(c, GRMHD_EUNSUPPORTED, "no digit-slice contraction in this context (contraction = 1)");
    DerivJob jb;
    jb.src = c->U[0]; jb.dst = c->scratch; jb.accumulate = 0; jb.pad = 0;
    CK(cudaMemcpyAsync(c->jobs + c->job_dbg, &jb, sizeof(jb), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->stream));
    CK(launch_contract_fx(dir, c->d, c->jobs + c->job_dbg, 1, c->fx_d[dir], dir == 0 ? c->fx_estride : 0, c->tc_err,
                          c->stream, 1));
    int te = 0;
    CK(cudaMemcpyAsync(&te, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!te) return GRMHD_OK;
    CK(cudaMemset(c->tc_err, 0, sizeof(int)));
    return set_err(c, GRMHD_ETIMEOUT, "a tensor-core contraction wait timed out (requested stall)");
}

extern "C" int grmhd_debug_theta(grmhd_ctx* c, const double* in, double* out, int nfields, const int* parity,
                                 int filter) {
    if (!c || !in || !out || !parity || nfields < 1 || (filter != 0 && filter != 1)) return GRMHD_EINVAL;
    const long long P = c->d.P;
    if (!c->ft) {
        if (nfields > 64) return GRMHD_EINVAL;
        std::vector<DerivJob> jb(nfields);
        for (int f = 0; f < nfields; f++) { jb[f].src = in + f * P; jb[f].dst = out + f * P; jb[f].accumulate = 0; jb[f].pad = 0; }
        CK(cudaMemcpyAsync(c->jobs + c->job_dbg, jb.data(), sizeof(DerivJob) * nfields, cudaMemcpyHostToDevice, c->stream));
        CK(contract(c, 1, filter, c->jobs + c->job_dbg, nfields));
        CK(cudaStreamSynchronize(c->stream));
        return GRMHD_OK;
    }
    if (nfields > c->nfold) return GRMHD_EINVAL;
    std::vector<FoldJob> fj(2 * (size_t)nfields);
    for (int f = 0; f < nfields; f++) {
        if (parity[f] != 1 && parity[f] != -1) return GRMHD_EINVAL;
        fj[f].src = in + f * P; fj[f].dst = c->Y + f * P; fj[f].parity = parity[f]; fj[f].accumulate = 0;
        FoldJob& u = fj[nfields + f];
        u.src = c->Z + f * P; u.dst = out + f * P; u.parity = parity[f]; u.accumulate = 0;
    }
    // the fold and unfold entries are contiguous blocks of nfold slots each
    CK(cudaMemcpyAsync(c->fjobs + c->fj_dbg, fj.data(), sizeof(FoldJob) * nfields, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->fjobs + c->fj_dbg_u, fj.data() + nfields, sizeof(FoldJob) * nfields, cudaMemcpyHostToDevice,
                       c->stream));
    CK(theta_fourier(c, filter, -1, c->fj_dbg, c->fj_dbg_u, nfields));
    CK(cudaStreamSynchronize(c->stream));
    return GRMHD_OK;
}

extern "C" const char* grmhd_strerror(int s) {
    switch (s) {
        case GRMHD_OK: return "ok";
        case GRMHD_EINVAL: return "invalid argument";
        case GRMHD_ENOMEM: return "out of memory";
        case GRMHD_ECUDA: return "CUDA runtime error";
        case GRMHD_ENAN: return "non-finite value in the evolved state";
        case GRMHD_ETIMEOUT: return "device-side wait timed out";
        case GRMHD_EUNSUPPORTED: return "option not supported by this library";
        case GRMHD_WPRECISION:
            return "warning: created; TF32 contractions (precision 2) exceed the mixed-precision error bar "
                   "(state L2 error O(1) after 100 steps on the 2-element workload); use precision 1";
        default: return "unknown status";
    }
}

extern "C" const char* grmhd_last_error(const grmhd_ctx* c) { return c ? c->err : "no context"; }

// ------------------------------------------------------------------ batch
#define BCK(call)                                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            snprintf(b->err, sizeof(b->err), "%s: %s", #call, cudaGetErrorString(e_)); \
            return GRMHD_ECUDA;                                                        \
        }                                                                              \
    } while (0)

extern "C" int grmhd_batch_create(int n, const grmhd_grid* grids, const grmhd_physics* phys,
                                  const grmhd_opts* opts, void* cuda_stream, grmhd_batch** out) {
    if (!out || n < 1 || !grids || !phys || !opts) return GRMHD_EINVAL;
    *out = nullptr;
    // every instance's parameters are checked before any device work
    {
        char msg[256] = {0};
        for (int i = 0; i < n; i++) {
            const int st = validate(&grids[i], &phys[i], &opts[i], msg);
            if (st != GRMHD_OK) return st;
        }
    }
    grmhd_batch* b = new (std::nothrow) grmhd_batch();
    if (!b) return GRMHD_ENOMEM;
    if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
    else {
        if (cudaStreamCreate(&b->stream) != cudaSuccess) { delete b; return GRMHD_ECUDA; }
        b->own_stream = true;
    }
    b->n = n;
    b->grp.assign(n, -1);
    b->idx.assign(n, -1);
    // group compatible instances (same node counts, theta range, EOS, floors, options)
    std::vector<std::vector<int>> members;
    for (int i = 0; i < n; i++) {
        int g = -1;
        for (size_t k = 0; k < members.size(); k++) {
            int f = members[k][0];
            if (same_group(grids[f], phys[f], grids[i], phys[i]) && std::memcmp(&opts[f], &opts[i], sizeof(grmhd_opts)) == 0) {
                g = (int)k;
                break;
            }
        }
        if (g < 0) { members.emplace_back(); g = (int)members.size() - 1; }
        b->grp[i] = g;
        b->idx[i] = (int)members[g].size();
        members[g].push_back(i);
    }
    b->ngroups = (int)members.size();
    b->groups = new (std::nothrow) grmhd_ctx*[b->ngroups]();
    if (!b->groups) { grmhd_batch_destroy(b); return GRMHD_ENOMEM; }
    for (int g = 0; g < b->ngroups; g++) {
        std::vector<grmhd_grid> gg;
        std::vector<grmhd_physics> pp;
        for (int i : members[g]) { gg.push_back(grids[i]); pp.push_back(phys[i]); }
        int st = ctx_create((int)gg.size(), gg.data(), pp.data(), &opts[members[g][0]], b->stream, &b->groups[g]);
        if (st) { grmhd_batch_destroy(b); return st; }
    }
    *out = b;
    for (int i = 0; i < n; i++)
        if (opts[i].precision == 2) return GRMHD_WPRECISION;   // created; see grmhd_create
    return GRMHD_OK;
}

extern "C" int grmhd_batch_num_groups(const grmhd_batch* b) { return b ? b->ngroups : -1; }

extern "C" long long grmhd_batch_num_points(const grmhd_batch* b, int i) {
    if (!b || i < 0 || i >= b->n) return -1;
    const grmhd_ctx* c = b->groups[b->grp[i]];
    return (long long)c->inst_E[b->idx[i]] * c->d.elem;
}

extern "C" int grmhd_batch_num_vars(const grmhd_batch* b, int i) {
    if (!b || i < 0 || i >= b->n) return -1;
    return b->groups[b->grp[i]]->nv;
}

extern "C" int grmhd_batch_coords(const grmhd_batch* b, int i, double* r, double* th, double* ph) {
    if (!b || i < 0 || i >= b->n) return GRMHD_EINVAL;
    const grmhd_ctx* c = b->groups[b->grp[i]];
    const int in = b->idx[i], off = c->inst_off[in];
    const Dims& d = c->d;
    for (int e = 0; e < c->inst_E[in]; e++)
        for (int ii = 0; ii < d.Nr; ii++)
            for (int k = 0; k < d.Nt; k++)
                for (int l = 0; l < d.Np; l++) {
                    size_t p = (((size_t)e * d.Nr + ii) * d.Nt + k) * d.Np + l;
                    if (r) r[p] = c->r_nodes[(size_t)(off + e) * d.Nr + ii];
                    if (th) th[p] = c->th_nodes[k];
                    if (ph) ph[p] = c->ph_nodes[l];
                }
    return GRMHD_OK;
}

extern "C" int grmhd_batch_init_prims(grmhd_batch* b, int i, const double* rho, const double* p,
                                      const double* vr, const double* vth, const double* vph,
                                      const double* A_phi) {
    if (!b || i < 0 || i >= b->n || !rho || !p || !vr || !vth || !vph || !A_phi) return GRMHD_EINVAL;
    grmhd_ctx* c = b->groups[b->grp[i]];
    std::vector<double> U;
    build_instance_state(c, b->idx[i], rho, p, vr, vth, vph, A_phi, U);
    return inst_set_state(c, b->idx[i], U.data(), 0);
}

extern "C" int grmhd_batch_set_state(grmhd_batch* b, int i, const double* state, int on_device) {
    if (!b || i < 0 || i >= b->n || !state) return GRMHD_EINVAL;
    return inst_set_state(b->groups[b->grp[i]], b->idx[i], state, on_device);
}

extern "C" int grmhd_batch_get_state(grmhd_batch* b, int i, double* state, int on_device) {
    if (!b || i < 0 || i >= b->n || !state) return GRMHD_EINVAL;
    grmhd_ctx* c = b->groups[b->grp[i]];
    return inst_copy(c, b->idx[i], c->U[0], c->nv, nullptr, state, on_device, 0);
}

extern "C" int grmhd_batch_cfl_dt(grmhd_batch* b, double* dt_out) {
    if (!b || !dt_out) return GRMHD_EINVAL;
    for (int k = 0; k < b->ngroups; k++) {
        grmhd_ctx* c = b->groups[k];
        BCK(launch_cfl(c->d, c->n_inst, c->U[0], c->hmin, c->opts.cfl, c->dt, c->lam_bits, b->stream));
        std::vector<double> dts(c->n_inst);
        BCK(cudaMemcpyAsync(dts.data(), c->dt, sizeof(double) * c->n_inst, cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        for (int i = 0; i < b->n; i++)
            if (b->grp[i] == k) dt_out[i] = dts[b->idx[i]];
    }
    return GRMHD_OK;
}

extern "C" long long grmhd_batch_launch_count(const grmhd_batch* b) { return b ? b->launches_per_step : -1; }

extern "C" int grmhd_batch_step(grmhd_batch* b, const double* dt, int nsteps) {
    NvtxRange nvtx_range("grmhd_batch_step");
    if (!b || !dt || nsteps < 1) return GRMHD_EINVAL;
    for (int i = 0; i < b->n; i++)
        if (!(dt[i] > 0.0)) return GRMHD_EINVAL;
    if (!b->gexec || b->g_nsteps != nsteps) {
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int st = GRMHD_OK;
        long long launches = 0;
        for (int s = 0; s < nsteps && st == GRMHD_OK; s++)
            for (int k = 0; k < b->ngroups && st == GRMHD_OK; k++) {
                b->groups[k]->launches_tmp = 0;
                st = enqueue_step(b->groups[k]);
                launches += b->groups[k]->launches_tmp;
            }
        b->launches_per_step = launches / nsteps;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (st) { if (g) cudaGraphDestroy(g); return st; }
        BCK(e);
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        BCK(e);
        b->g_nsteps = nsteps;
    }
    for (int k = 0; k < b->ngroups; k++) {
        grmhd_ctx* c = b->groups[k];
        std::vector<double> dts(c->n_inst);
        for (int i = 0; i < b->n; i++)
            if (b->grp[i] == k) dts[b->idx[i]] = dt[i];
        BCK(cudaMemcpyAsync(c->dt, dts.data(), sizeof(double) * c->n_inst, cudaMemcpyHostToDevice, b->stream));
    }
    BCK(cudaGraphLaunch(b->gexec, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return GRMHD_OK;
}

extern "C" int grmhd_batch_destroy(grmhd_batch* b) {
    if (!b) return GRMHD_EINVAL;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->groups) {
        for (int g = 0; g < b->ngroups; g++)
            if (b->groups[g]) grmhd_destroy(b->groups[g]);
        delete[] b->groups;
    }
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return GRMHD_OK;
}

extern "C" const char* grmhd_batch_last_error(const grmhd_batch* b) { return b ? b->err : "no batch"; }
