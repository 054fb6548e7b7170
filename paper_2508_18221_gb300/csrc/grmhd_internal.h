// Internal declarations shared by the library's translation units (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/grmhd.h"

namespace gk {

// canonical variable slots
enum {
    NV = 32,
    V_GT = 0, V_PHI = 6, V_AT = 7, V_K = 13, V_GAM = 14, V_ALPHA = 17, V_BETA = 18, V_BG = 21,
    V_D = 24, V_S = 25, V_TAU = 28, V_B = 29, N_BSSN = 24, N_VAL = 8,
    V_PSI = 32, NV_MAX = 33,   // GLM scalar (glm = 1: 33 variables)
    // differentiated fields: canonical variables 0..20 (all BSSN + gauge but B^i)
    N_D1 = 21,
    // second derivatives of gammatilde_ij (0..5), phi (6), alpha (17), beta^i (18..20)
    N_D2 = 11,
    N_PRIM = 7,     // rho, v^r, v^th, v^ph, eps, p, W
    N_FLUX = 24,    // sqrt(gamma) scriptF^i_v  [dir][var]
    N_TMN = 10,     // T^{00},T^{01},T^{02},T^{03},T^{11},T^{12},T^{13},T^{22},T^{23},T^{33}
};

// d1 field f (0..20) direction d: index (f*3 + d); d2 field slot s (0..10) pair q:
// (s*6 + q) with q = rr, rth, rph, thth, thph, phph
__host__ __device__ inline int d2_slot_of_var(int v) {
    return v <= 6 ? v : (v >= 17 && v <= 20 ? v - 10 : -1);
}

struct Dims {
    int E, Nr, Nt, Np;
    long long P;          // points
    long long NtNp;       // points per radial shell
    long long elem;       // points per element
    // element topology of a group of instances concatenated along r (device pointers)
    const unsigned char* iface_next;  // [E] 1: element e is coupled to e + 1
    const int* elem_inst;             // [E] instance owning element e
};

struct PhysParams {
    double M, a, gam, rho_atm, eps_atm;
    double eta;
    int gauge, evolve_metric;
    int evolve_fluid;     // 0: Valencia right-hand side zero (BSSN half of a split step)
    int glm;              // 1: GLM cleaning with psi (variable 32)
    double glm_ch2, glm_itau;
    int c2p_maxit;
    double c2p_tol;
    double c2p_lambda;    // > 0: the paper's damped iteration with this initial damping
    double w_end;         // Clenshaw-Curtis end weight on [-1, 1] for n_r CGL nodes
};

struct DerivJob {
    const double* src;
    double* dst;
    int accumulate;       // 0: dst = D src, 1: dst += D src
    int pad;
};

// tensor-core contraction job: src is double (state, fluxes) or float (first derivatives)
struct TcJob {
    const void* src;
    float* dst;
    int accumulate;
    int pad;
};

// Fourier theta basis: one field of a fold (src = canonical field, dst = folded pair of
// halves) or unfold (src = folded contraction result, dst = canonical field) pass; double
// or float values as the launch says; parity +1 / -1 of the field under the extension
struct FoldJob {
    const void* src;
    void* dst;
    int parity;
    int accumulate;       // unfold only: 0 dst = result, 1 dst += result
};

// ---- kernel launchers (defined in kernels_*.cu); all return cudaGetLastError()
// one-time function-attribute setup (shared-memory opt-in); call outside stream capture
cudaError_t kernels_init();
cudaError_t eo_init();
cudaError_t tc_init();
// met: 9 P doubles written per node (e^{4phi}, e^{-4phi}, sqrt(gamma), gammatilde^ij in the
// packed order rr r-theta r-phi theta-theta theta-phi phi-phi), read by launch_rhs
cudaError_t launch_prep(const Dims& d, const PhysParams& pp, const double* U, double* prim,
                        double* flux, double* tmn, double* lam, unsigned long long* nfail, double* met,
                        cudaStream_t s, int fp32_algebra = 0);
struct RKCoef { double a, b, c, w; int acc_mode; };  // out = a U0 + b Us + c dt L (+acc)
// d1, d2, divF are double (FP64 mode) or float (deriv_fp32 = 1, mixed modes); ham != null
// also writes the Hamiltonian constraint per node (diagnostics)
cudaError_t launch_rhs(const Dims& d, const PhysParams& pp, const double* U0, const double* Us,
                       const double* prim, const double* flux, const double* tmn,
                       const double* lam, const double* met, const void* d1, const void* d2,
                       const void* divF, const void* divB, int deriv_fp32, const double* r_scale_dev,
                       const double* dt_dev, RKCoef co, double* out, double* acc, cudaStream_t s,
                       double* ham = nullptr);
// tensor-core contraction (kernels_tc.cu); op_img in the kernel's shared-memory layout
cudaError_t launch_contract_tc(int dir, int in_fp32, const Dims& d, const TcJob* jobs, int njobs,
                               const uint8_t* op_img, int tf32, const double* r_scale, int* err,
                               cudaStream_t s);
// FP64-accurate contraction on the FP16 tensor cores (kernels_fx.cu): exact digit
// slices of the FP64 values; op_img from fx_operator_image, img_estride = bytes between
// per-element images (radial direction) or 0; Np, Kp, KC from fx_geometry
void fx_geometry(int N, int* Np, int* Kp, int* KC);
bool fx_supported(int dir, int N);   // 2..128 nodes (even in phi)
cudaError_t fx_init();
// stall = 1 (test of the wait limits only): the tiles are never staged, so every wait of the
// kernel runs out (about 0.5 s), the CTAs leave and *err is set.  kind: 0 derivative, 1
// filter (the key of the tuning table; the arithmetic is the same).  tsets: TMEM accumulator
// sets (1, or 2: the next item's MMAs run while the epilogue drains the previous one; one
// CTA per SM); 0 takes the tuning table's choice for the class
cudaError_t launch_contract_fx(int dir, const Dims& d, const DerivJob* jobs, int njobs, const uint8_t* op_img,
                               long long img_estride, int* err, cudaStream_t s, int stall = 0, int kind = 0,
                               int tsets = 0);
// tuning table of the digit-slice contraction (process-wide): accumulator sets per
// (direction, nodes, kind); 0 when the class was not tuned
void fx_tune_set(int dir, int N, int kind, int tsets);
int fx_tune_get(int dir, int N, int kind);
bool fx_two_sets_possible(int dir, int N);
cudaError_t launch_deriv(int dir, const Dims& d, const DerivJob* jobs_dev, int njobs,
                         const double* mat_dev, const double* r_scale_dev, cudaStream_t s);
// reflection-split contraction (kernels_eo.cu): cudaErrorNotSupported when N has no
// compiled instance; sign -1 for derivatives, +1 for filters
bool eo_supported(int dir, int N);
cudaError_t launch_deriv_eo(int dir, const Dims& d, const DerivJob* jobs, int njobs,
                            const double* op_split, int sign, const double* r_scale,
                            cudaStream_t s);
cudaError_t launch_iface_avg(const Dims& d, double* base, long long field_stride, int nfields,
                             cudaStream_t s);
// Fourier theta: fold the phi pairs (l, l + N_phi/2) of every job's field into two halves
// [E][Nr][Nt][N_phi/2] (first the half the even extension operator takes), and the
// inverse; d are the full grid's dims; fp32 selects float values
cudaError_t launch_theta_fold(const Dims& d, const FoldJob* jobs, int njobs, int fp32, cudaStream_t s);
cudaError_t launch_theta_unfold(const Dims& d, const FoldJob* jobs, int njobs, int fp32, cudaStream_t s);
cudaError_t launch_iface_avg_f(const Dims& d, float* base, long long field_stride, int nfields,
                               cudaStream_t s);
// per instance: dt[i] = cfl * hmin[i] / max over its nodes of lambda
cudaError_t launch_cfl(const Dims& d, int n_inst, const double* U, const double* hmin_dev, double cfl,
                       double* dt_dev, unsigned long long* lam_bits, cudaStream_t s);
cudaError_t launch_diag(const Dims& d, const PhysParams& pp, const double* U,
                        const double* prim, const double* wq, const double* divB,
                        double* out_dev, cudaStream_t s, const double* ham = nullptr);
cudaError_t launch_nan_check(long long n, const double* U, int* flag, cudaStream_t s);

// Approximate XCTS initial data (kernels_xcts.cu): operators of the boundary-value problem
// on one instance's grid (Fourier theta basis) and the fixed-point solve
struct XctsOps {
    int E, Nr, Nt, Np;
    std::vector<double> Dr, Drr;   // [E][Nr][Nr] element radial first / second derivative
    std::vector<double> D1, D2;    // [2][Nt][Nt] theta first / second derivative, mode parity +1, -1
    std::vector<double> r, th;     // [E * Nr] radial nodes, [Nt] theta nodes
    double M, r_min, r_max;
};
// psi_host: initial guess in, solution out (num_points values); changes (iters entries, may
// be null): max |psi_{k+1} - psi_k|; stats (may be null): set-up ms (Schur forms + inverses),
// mean ms per iteration, iterations done; returns a GRMHD status, message in msg
int xcts_solve(const XctsOps& o, const double* rho_host, double* psi_host, int iters, double tol,
               double* changes, double* stats, cudaStream_t s, char* msg, size_t msglen);

}  // namespace gk
