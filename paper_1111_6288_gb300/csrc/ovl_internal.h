// Internal declarations of libovl: data layouts, kernel launchers, host helpers.
//
// Internal layouts (all site-major over the fastest index so that a warp reads
// 32 consecutive sites of one component; component k = 3*spin + colour):
//   FP64 spinor  [rhs][12][V] double2
//   FP32 spinor  [rhs][6][V]  float4 = components (2q, 2q+1); spins 0,1 are planes 0-2
//   FP64 links   [4][9][V]    double2, entry 3*a + b of U_mu(n)
//   FP32 links   [4][3][V]    float4 = rows 0 and 1 of U_mu(n); row 2 = conj(row0 x row1)
//   FP16 / BF16  spinors [rhs][3][V] uint4 (+ a float scale per site for FP16) and links
//                rows 0 and 1 in 24 bytes, FP32 arithmetic (half_store.h)
//   bank         [n_ev][...]  the spinor layout of its precision
// A spinor vector is 12 V complex numbers (192 B or 96 B per site) in both precisions,
// so element-wise kernels and inner products treat vectors as flat complex arrays.
#pragma once

#include <cuda_runtime.h>

#include "half_store.h"

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

namespace ovl {

// Number of kernels this library has launched (all contexts, all streams).
extern std::atomic<long long> g_launches;
inline void count_launch(long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

template <typename R> struct C2;
template <> struct C2<double> { typedef double2 T; };
template <> struct C2<float> { typedef float2 T; };

// Arithmetic type of a storage type: itself for FP64 and FP32, FP32 for the 16-bit formats.
template <typename S> struct Arith { typedef S type; };
template <> struct Arith<H16> { typedef float type; };
template <> struct Arith<B16> { typedef float type; };

// Lattice geometry and boundary factors (1 periodic, -1 antiperiodic, 0 Dirichlet).
struct Geom {
    int L[4];       // Lx, Ly, Lz, Lt
    int V;          // sites
    double bcf[4];  // boundary factor per direction
};

// Epilogue of a Wilson application (all coefficients uniform over right-hand sides):
//   z   = c_op * H_w(in) + c1 * v1
//   z   = gamma5 z                          if g5
//   z   = chi_j * P_{chi_j} z               if chi && chi[j] != 0  (P_+- = (1 +- gamma5)/2)
//   out = z + c2 * v2 + c3 * v3
// Null vectors contribute nothing.  v3 may alias out (read and written by the same thread).
struct Epilogue {
    double c_op = 1.0;
    double c1 = 0.0, c2 = 0.0, c3 = 0.0;
    const void* v1 = nullptr;
    const void* v2 = nullptr;
    const void* v3 = nullptr;
    int g5 = 0;
    const signed char* chi = nullptr;  // device [nrhs]
    const double* c2r = nullptr;       // device: c2 of rhs j is c2 * c2r[j * c2r_stride] if set
    long long c2r_stride = 0;
};

// ---- kernels: dslash.cu ---------------------------------------------------
// S: storage type (double, float, H16, B16; the 16-bit ones compute in FP32).
// deriv: apply dH_w/dphi (the phi-derivative of the x hops, per right-hand-side phase) in
// place of H_w; the epilogue is the same.  shape: right-hand sides per thread block in the
// low bits (1, 2, 4 or 8; 0 = default), | kShapeDense for the FP32 kernel whose registers allow
// 7 resident blocks per SM instead of 6 (no effect in FP64).
// | kShapeTiled: the FP32 / 16-bit kernel that stages whole x-rows in shared memory (lattices
// for which tile_rows() > 0; otherwise the plain kernel runs).
constexpr int kShapeRhsMask = 15;
constexpr int kShapeDense = 16;
constexpr int kShapeTiled = 32;
// Rows of x per block of the tiled kernel for `by` right-hand sides per block (0: not tileable).
int tile_rows(const Geom& g, int by);
// 1 if a bounded device wait ran out since the last call (and clears it), 0 if not, -1 on error.
int take_wait_timeouts();
// One block waiting on an mbarrier nothing completes, for limit_cycles: sets the timeout flag.
void launch_bounded_wait_selftest(long long limit_cycles, cudaStream_t s);
template <typename R>
void launch_dslash(const Geom& g, double m0, const void* links, const void* in, void* out, int nrhs,
                   const double* d_phase, const Epilogue& e, cudaStream_t s, bool deriv = false,
                   int shape = 0);

// ---- kernels: blas.cu -----------------------------------------------------
// ABI spinor [rhs][site][12] (dtype_in: 0 complex128, 1 complex64) -> internal [rhs][12][V] of R.
template <typename R>
void launch_pack_spinor(const void* abi, int dtype_in, void* internal, int V, int nrhs, cudaStream_t s);
template <typename R>
void launch_unpack_spinor(const void* internal, void* abi, int dtype_out, int V, int nrhs, cudaStream_t s);
// ABI links [4][site][3][3] -> internal links of R (FP64: [4][9][V] with the antiperiodic
// boundary signs of g folded in; FP32: [4][3][V] float4, rows 0 and 1).
template <typename R>
void launch_pack_gauge(const void* abi, int dtype_in, void* internal, const Geom& g, cudaStream_t s);
// Conversion of nvec spinor vectors between precisions (and internal layouts).
template <typename RI, typename RO>
void launch_convert(const void* in, void* out, int V, long long nvec, cudaStream_t s);
// FP32 spinors -> 16-bit storage S (times factor, then rounded), and back.
template <typename S>
void launch_to_half(const void* in32, void* out, int V, long long nvec, double factor, cudaStream_t s);
template <typename S>
void launch_from_half(const void* in, void* out32, int V, long long nvec, cudaStream_t s);
// ABI links -> 16-bit storage S (rows 0 and 1).
template <typename S>
void launch_pack_gauge_half(const void* abi, int dtype_in, void* internal, int V, cudaStream_t s);

// Per-rhs reductions over n complex numbers each (vectors at stride n).  Results are
// written to host memory after an internal synchronisation of s.  Deterministic.
template <typename R>
void dot_rhs(const void* a, const void* b, long long n, int nrhs, double2* host_out, double2* d_partial,
             double2* d_out, cudaStream_t s);
template <typename R>
void norm2_rhs(const void* a, long long n, int nrhs, double* host_out, double2* d_partial, double2* d_out,
               cudaStream_t s);

// y_j = a_j x_j + b_j y_j for per-rhs real scalars (host arrays of length nrhs <= kMaxRhs).
constexpr int kMaxRhs = 256;
template <typename R>
void launch_axpby(const double* a, const void* x, const double* b, void* y, long long n, int nrhs, cudaStream_t s);
// CG step: x_j += alpha_j p_j; r_j -= alpha_j Ap_j.
template <typename R>
void launch_cg_xr(const double* alpha, const void* p, const void* Ap, void* x, void* r, long long n, int nrhs,
                  cudaStream_t s);
// Scale by a complex scalar per rhs is not needed; plain scale by a uniform real:
template <typename R>
void launch_scale(double a, const void* x, void* y, long long n, cudaStream_t s);
// y = P_chi x per rhs (chi in {+1,-1}; spins 0,1 for +1, 2,3 for -1), V sites, rhs mapping
// out rhs j <- in rhs src[j].
template <typename R>
void launch_chiral_split(const void* x, void* y, const int* src, const signed char* chi, int V, int nsys,
                         cudaStream_t s);
// y = gamma5 x.
template <typename R>
void launch_gamma5(const void* x, void* y, int V, int nrhs, cudaStream_t s);

// C[i][j] = <A_i, B_j> over n complex numbers; A_i at A + i*strideA, B_j at B + j*strideB
// (strides in complex elements).  C: device double2 [na][nb] (row-major), deterministic.
template <typename R>
void multidot(const void* A, long long strideA, int na, const void* B, long long strideB, int nb, long long n,
              double2* d_C, double2* d_partial, long long partial_cap, cudaStream_t s);
// out_j = alpha * X_j + sum_i A_i C[i][j] for j < nb; C is device double2 [na][ldc] (column j).
template <typename R>
void combine(const void* A, long long strideA, int na, const double2* d_C, int ldc, int nb, double alpha,
             const void* X, long long strideX, void* out, long long strideO, long long n, cudaStream_t s);

// Small-space projection of nb vectors X (each n complex, stride n) on na bank vectors V:
// C = V^+ X (device, [na][min(nb,4)] per group of 4), Xp = X - V C, Ys = V diag(signs) C.
// Reads V twice per group of 4 right-hand sides.  na <= 384.
template <typename R>
void small_space_project(const void* V, int na, const double* d_signs, const void* X, int nb, void* Xp, void* Ys,
                         long long n, double2* d_C, double2* d_partial, long long partial_cap, cudaStream_t s);

// ---- tensor-core projection: proj_tc.cu --------------------------------------------------
// The same projection as small_space_project for FP32 vectors on the tcgen05 tensor cores (TF32 with
// the three-term split, FP32-accurate): C = V^+ X by a split-K GEMM (partials in d_partial, at least
// 152 x na x min(nb, 32) double2), then X - V C and V diag(s) C; groups of up to 32 right-hand sides.
// d_img: tc_project_image_bytes(na) bytes of scratch for the pre-split coefficients.  na <= kTcMaxBank.
constexpr int kTcMaxBank = 384;
size_t tc_project_image_bytes(int na);
bool tc_project_available();
cudaError_t small_space_project_tc(const void* V, int na, const double* d_signs, const void* X, int nb, void* Xp,
                                   void* Ys, long long n, double2* d_C, double2* d_partial, long long partial_cap,
                                   void* d_img, cudaStream_t s);
// 1 if a bounded wait of a tensor-core kernel ran out since the last call (and clears it), else 0; -1 on error.
int take_tc_timeouts();

// Partial-sum buffer size (double2 elements) needed by dot_rhs/norm2_rhs.
constexpr int kRedBlocks = 608;

// Message returned by ov_last_error(NULL) (errors of calls that have no context).
void set_global_error(const char* msg);

// ---- host linear algebra: hostla.cpp --------------------------------------
// Column-major complex matrices as std::vector<double2>-compatible arrays of (re, im).
struct HostCplx { double re, im; };
// Cholesky A = L L^+ (lower); returns false if not positive definite.
bool host_cholesky(int n, std::vector<HostCplx>& A);
// Inverse of the conjugate transpose of a lower-triangular L: returns R = L^{-+} (upper).
void host_inv_lower_dag(int n, const std::vector<HostCplx>& L, std::vector<HostCplx>& R);
// Eigen-decomposition of a Hermitian matrix (cyclic Jacobi): A = Z diag(w) Z^+,
// eigenvalues ascending. A is overwritten.
void host_eigh(int n, std::vector<HostCplx>& A, std::vector<double>& w, std::vector<HostCplx>& Z);
// Chebyshev interpolant coefficients of x^{-1/2} on [eps, 1] (c_0 halved).
void host_chebyshev_coeffs(int n, double eps, double* out);
// The same for 1/(a + sqrt(x)), a > 0.
void host_chebyshev_coeffs_shifted_inverse_root(int n, double eps, double a, double* out);
// delta = max over [eps, 1] of |1 - sqrt(x) P(x)| for P = sum_k coeffs[k] T_k(y) (Sec. 2, eq. 2),
// on a grid of 4097 points uniform in the Chebyshev angle.
double host_poly_delta(const double* coeffs, int n, double eps);
// The degree-n polynomial of least relative error |1 - sqrt(x) P(x)| on [eps, 1] (Remez exchange),
// in the same basis; returns its delta.
double host_minimax_coeffs(int n, double eps, double* out);

}  // namespace ovl
