// Host-side operators and initial data (see host_ops.cpp).
#pragma once
#include <cstdint>
#include <vector>

namespace gk {
std::vector<double> cgl_nodes(int n);
std::vector<double> gauss_nodes(int n);
std::vector<double> cheb_lobatto_D(int n);      // d/dx on ascending CGL nodes of [-1, 1]
std::vector<double> cheb_gauss_D(int n);        // d/dx on ascending Gauss nodes of [-1, 1]
std::vector<double> fourier_D_row(int n);       // circulant row of d/dphi, N even
std::vector<double> cheb_filter_matrix(int n, bool lobatto, double alpha, double p);
std::vector<double> fourier_filter_row(int n, double alpha, double p, bool dealias);
std::vector<double> quad_weights(int n, bool lobatto);
// Fourier theta basis: the n x n operators A + B (even) and A - B (odd) that act on the
// phi-pair sums and differences of the double-Fourier extension (host_ops.cpp), for the
// circulant row c of the 2n extended nodes (derivative or filter), times scale
void theta_extension_ops(const std::vector<double>& c, int n, std::vector<double>* even,
                         std::vector<double>* odd, double scale = 1.0);
// reflection-split packing [E | O | C | F | G] of a dense N x N operator (kernels_eo.cu);
// kind 0 Chebyshev node set, 1 Fourier node set
std::vector<double> split_operator(const std::vector<double>& M, int N, int kind);
std::vector<double> circulant(const std::vector<double>& row);
// operator D (N x N, row = output node) in the tensor-core kernel's shared-memory image:
// K-major core-matrix layout padded to 16 in both dims; 3 BF16 slices or 1 TF32 copy
std::vector<uint8_t> tc_operator_image(const std::vector<double>& D, int N, int tf32);
// operator scale * D (N x N) for the FP64-accurate tensor-core contraction
// (kernels_fx.cu): per K chunk of KC columns one tall FP16 matrix in the K-major
// core-matrix layout whose rows are, per pass of Npp = min(Np, 64) output rows, the seven
// balanced base-256 digit slices of those rows one after the other (each digit an FP16
// integer in [-128, 127]); then the Np row exponents (int32); size a multiple of 16 bytes
std::vector<uint8_t> fx_operator_image(const std::vector<double>& D, int N, double scale, int Np, int Kp,
                                       int KC);
// BSSN variables 0..23 of the Kerr-Schild slice at (r, theta)
void ks_bssn_point(double M, double a, double r, double th, double out[24]);
void prim_to_cons_point(double rho, double p, const double v_u[3], const double B_u[3],
                        const double g[3][3], double gam_eos, double* D, double S_d[3],
                        double* tau);
void metric_from_bssn_point(const double* bssn, double g[3][3], double* sqg);
// real Schur form of a real n x n row-major matrix with a real spectrum (host_eig.cpp):
// A = Q T Q^T with Q orthogonal and T upper triangular (both row-major n x n); *resid (may
// be null) max |Q T Q^T - A| / max |A|; false on a complex pair, no convergence or a
// residual above 1e-11
bool real_schur(int n, const double* A, double* Q, double* T, double* resid);
}  // namespace gk
