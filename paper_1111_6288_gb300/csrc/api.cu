// libovl C ABI: context, operator applications, small space, solver, eigensolver.
//
// Host orchestration of the kernels in dslash.cu and blas.cu.  Paper mapping:
//   apply_wilson          Sec. 2, H_w = gamma5 D_w
//   apply_sign_Hw         Sec. 2, sign(H_w) ~ V diag(s) V^+ + Q P(Q^2)(1 - V V^+)
//   apply_overlap         Sec. 2, eq. 1, D_ov = 1 + gamma5 sign(H_w); D(m) = (1 - m/2) D_ov + m
//   deflate               Sec. 2, small space from eigenvectors of Q
//   ov_eigensolve_Q       Sec. 3.1, low eigenmodes of H_w with Chebyshev acceleration
//   solve_overlap         Sec. 3.2, CG for D^{-1} psi, single precision late in the solve, adaptive
//                         polynomial order, deflation with the low modes of D_ov
//   solve_overlap_multimass  Sec. 3.2, multi-mass CG: a multi-shift CG cycle shared by the masses,
//                         then the cycles of solve_overlap per mass
//   ov_eigensolve_overlap Sec. 3.1-3.2, the D_ov low modes of one chiral sector (Lanczos)
//   ov_create (poly_kind) Sec. 2, eq. 2, Chebyshev interpolant or minimax polynomial of x^{-1/2}
//   ov_apply_dDdphi, ...  Sec. 4, derivatives with respect to the background field
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ovl.h"
#include "ovl_internal.h"

using namespace ovl;

namespace {

thread_local std::string g_create_error;

struct Bank {
    double phase = 0.0;
    int n = 0;
    void* V64 = nullptr;  // [n][12][V] double2
    void* V32 = nullptr;  // [n][12][V] float2
    double* d_signs = nullptr;  // [n]
    std::vector<double> signs;
    std::vector<double> theta;  // eigenvalues of Q
    // derivative data with respect to the field phase (built on first use)
    bool dready = false;
    void* Uh64 = nullptr;           // [n][12][V] double2: low-high vectors u_i
    std::vector<double2> M;         // [n][n] low-low block F[l_i, l_j] (V^+ dH V)_ij, row-major
};

struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Low modes of D_ov for the CG deflation of the solver (Sec. 3.2): Ritz pairs of the chiral-sector
// operator A0 = P_s [2 (1 + s sign(H_w))] P_s = P_s D_ov^+ D_ov P_s at one field phase.  The inner
// CG's operator at mass m is A(m) = (1 - m^2/4) A0 + m^2 on the sector, so one space serves every
// mass.  FP32 vectors in the internal layout.
struct DefSpace {
    double phase = 0.0;
    int chi = 1;
    int n = 0;
    void* W = nullptr;    // [n] orthonormal vectors of sector chi
    void* AW0 = nullptr;  // A0 W
    void* AWm = nullptr;  // A(m) W for the mass below
    double mass = -1.0;   // mass of AWm and Einv (-1: not prepared)
    std::vector<HostCplx> Einv;  // (W^+ A(m) W)^{-1}, n x n column-major
    std::vector<double> theta, res;  // Ritz values of A0 and residual norms |A0 w - theta w|
    // FP64: W itself and D_ov^+ W, so that the solver adds the space's share of its correction,
    // D(m)^+ W c, in FP64; DmW = D(m)^+ W for the mass dm_mass
    void* W64 = nullptr;
    void* DW64 = nullptr;
    void* DmW64 = nullptr;
    double dm_mass = -1.0;
    // FP64 A0 W = 2 P_s D_ov^+ W (W lies in sector s, so gamma5 W = s W), A(m) W and
    // (W^+ A(m) W)^{-1} in FP64: the solver takes the space's part of each sector residual with
    // these before the FP32 CG sees it
    void* AW64 = nullptr;
    void* AWm64 = nullptr;
    std::vector<HostCplx> Einv64;
};

}  // namespace

struct ov_ctx {
    Geom g;
    ov_params p;
    std::vector<double> coeffs;
    double hw_norm = 0.0;
    double delta = 0.0;  // max over [eps, 1] of |1 - sqrt(x) P(x)| (Sec. 2, eq. 2)
    bool custom_coeffs = false;  // the caller gave the coefficients (no lower-degree polynomials)
    // lower-degree polynomials of the context's kind on the same interval and their delta, by degree
    std::map<int, std::vector<double>> coeff_sets;
    std::map<int, double> delta_of;
    std::string err;
    std::string info;  // summary of the last eigensolver / solve call
    void* U64 = nullptr;
    void* U32 = nullptr;
    void* U16 = nullptr;  // 16-bit links of an FP16 / BF16 context
    bool gauge_set = false;
    std::vector<Bank> banks;
    std::vector<DefSpace> dspaces;  // D_ov deflation spaces per (phase, chirality)
    std::map<std::string, Buf> ws;
    double2* d_partial = nullptr;
    long long partial_cap = 0;
    double2* d_red = nullptr;
    double2* d_C = nullptr;   // small matrices [cap_c]
    double2* d_C2 = nullptr;
    long long cap_c = 0;
    double* d_phase = nullptr;  // per-system phases
    signed char* d_chi = nullptr;
    int* d_idx = nullptr;
    int cap_sys = 0;
    long long dslash_count = 0;
    long long sign_count = 0;
    long long cg_stalls = 0;  // inner-CG systems stopped at a stalled residual (16-bit storage)
    // optional CUDA-event timing of the Clenshaw loops (the Wilson kernels of the polynomial)
    // CUDA graphs of the Clenshaw loop, keyed by precision, systems and buffers
    bool use_graphs = true;
    // autotuned right-hand sides per Wilson-kernel block, keyed by precision and systems
    std::map<std::pair<int, int>, int> launch_shape;
    // small-space projection of FP32 vectors: 0 = timed per (bank size, batch), 1 = CUDA cores,
    // 2 = tensor cores; the timed choice per (bank size, batch)
    int proj_method = 0;
    std::map<std::pair<int, int>, int> proj_choice;
    // working-set budget of the eigensolver's chunked passes (filter recurrence, residuals)
    long long eig_chunk_bytes = 16000000000LL;
    Buf tc_img;  // pre-split coefficients of the tensor-core projection
    std::string tune_log;
    cudaStream_t cap_stream = nullptr;
    std::map<std::string, std::pair<cudaGraphExec_t, void*>> graphs;  // exec, buffer holding p
    bool profile = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[4];  // per OV_PREC_* of the recurrence
    long long prof_launches[4] = {0, 0, 0, 0};
    double prof_bytes[4] = {0.0, 0.0, 0.0, 0.0};
};

namespace {

int fail(ov_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return code;
}

#define CK(call)                                                                                          \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail(c, OV_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                           \
    } while (0)
#define CKL()                                                                                           \
    do {                                                                                                \
        cudaError_t e_ = cudaGetLastError();                                                            \
        if (e_ != cudaSuccess)                                                                          \
            return fail(c, OV_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__,    \
                        __LINE__);                                                                      \
    } while (0)
#define TRY(x)                    \
    do {                          \
        int rc_ = (x);            \
        if (rc_ != OV_OK) return rc_; \
    } while (0)

template <typename R>
constexpr int prec_of() {
    return std::is_same<R, double>::value ? OV_PREC_F64
           : std::is_same<R, float>::value ? OV_PREC_F32
           : std::is_same<R, H16>::value   ? OV_PREC_F16
                                           : OV_PREC_BF16;
}

// bytes of one spinor vector, and of one site's spinor and links, per precision
size_t vec_bytes(const ov_ctx* c, int prec) {
    if (prec == OV_PREC_F16) return (size_t)half_rhs_bytes<H16>(c->g.V);
    if (prec == OV_PREC_BF16) return (size_t)half_rhs_bytes<B16>(c->g.V);
    return (size_t)12 * c->g.V * (prec == OV_PREC_F64 ? 16 : 8);
}
double site_spinor_bytes(int prec) { return prec == OV_PREC_F64 ? 192 : prec == OV_PREC_F32 ? 96 : prec == OV_PREC_F16 ? 52 : 48; }
double site_link_bytes(int prec) { return prec == OV_PREC_F64 ? 576 : prec == OV_PREC_F32 ? 192 : 96; }


// Named workspace of at least nvec spinor vectors of the given precision.
int workspace(ov_ctx* c, const std::string& name, int prec, long long nvec, void** out) {
    const size_t need = vec_bytes(c, prec) * (size_t)std::max<long long>(nvec, 1);
    static const char* suffix[4] = {"/64", "/32", "/16", "/b16"};
    const std::string key = name + suffix[prec];
    Buf& b = c->ws[key];
    if (b.bytes < need) {
        if (b.ptr) {
            CK(cudaDeviceSynchronize());
            CK(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&b.ptr, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, OV_ERR_OOM, "workspace '%s': cudaMalloc(%zu) failed: %s", key.c_str(), need,
                        cudaGetErrorString(e));
        }
        b.bytes = need;
    }
    *out = b.ptr;
    return OV_OK;
}

// Free the named workspaces whose names start with prefix (after the stream's work is done).
int release_workspaces(ov_ctx* c, const std::string& prefix, cudaStream_t s) {
    CK(cudaStreamSynchronize(s));
    for (auto it = c->ws.begin(); it != c->ws.end();) {
        if (it->first.compare(0, prefix.size(), prefix) == 0) {
            if (it->second.ptr) CK(cudaFree(it->second.ptr));
            it = c->ws.erase(it);
        } else {
            ++it;
        }
    }
    return OV_OK;
}

// The same after a failed call: the stream's error (already reported) is not checked again, and the
// buffers leave the context even if freeing them fails.
void release_workspaces_after_error(ov_ctx* c, const std::string& prefix, cudaStream_t s) {
    cudaStreamSynchronize(s);
    for (auto it = c->ws.begin(); it != c->ws.end();) {
        if (it->first.compare(0, prefix.size(), prefix) == 0) {
            if (it->second.ptr) cudaFree(it->second.ptr);
            it = c->ws.erase(it);
        } else {
            ++it;
        }
    }
}

int ensure_small(ov_ctx* c, long long nmat, long long npartial, int nsys) {
    if (nmat > c->cap_c) {
        if (c->d_C) {
            CK(cudaDeviceSynchronize());
            CK(cudaFree(c->d_C));
            CK(cudaFree(c->d_C2));
        }
        c->cap_c = std::max<long long>(nmat, 4096);
        CK(cudaMalloc(&c->d_C, sizeof(double2) * c->cap_c));
        CK(cudaMalloc(&c->d_C2, sizeof(double2) * c->cap_c));
    }
    if (npartial > c->partial_cap) {
        if (c->d_partial) {
            CK(cudaDeviceSynchronize());
            CK(cudaFree(c->d_partial));
        }
        c->partial_cap = std::max<long long>(npartial, 1 << 20);
        CK(cudaMalloc(&c->d_partial, sizeof(double2) * c->partial_cap));
    }
    if (nsys > c->cap_sys) {
        if (c->d_phase) {
            CK(cudaDeviceSynchronize());
            CK(cudaFree(c->d_phase));
            CK(cudaFree(c->d_chi));
            CK(cudaFree(c->d_idx));
            CK(cudaFree(c->d_red));
        }
        c->cap_sys = std::max(nsys, 64);
        CK(cudaMalloc(&c->d_phase, sizeof(double) * c->cap_sys));
        CK(cudaMalloc(&c->d_chi, c->cap_sys));
        CK(cudaMalloc(&c->d_idx, sizeof(int) * 2 * c->cap_sys));
        CK(cudaMalloc(&c->d_red, sizeof(double2) * c->cap_sys));
    }
    return OV_OK;
}

// links stored for storage type S
template <typename S>
const void* links_of(const ov_ctx* c) {
    if constexpr (std::is_same<S, double>::value) return c->U64;
    else if constexpr (std::is_same<S, float>::value) return c->U32;
    else return c->U16;
}

Bank* find_bank(ov_ctx* c, double phase) {
    for (auto& b : c->banks)
        if (b.phase == phase) return &b;
    return nullptr;
}

// Coefficients of the degree-n polynomial of the context's kind (interpolant or minimax) on its
// interval (n = poly_degree: the context's own, which may be the caller's).
const std::vector<double>& coeffs_of(ov_ctx* c, int n) {
    if (n == c->p.poly_degree) return c->coeffs;
    auto it = c->coeff_sets.find(n);
    if (it == c->coeff_sets.end()) {
        std::vector<double> cf(n + 1);
        if (c->p.poly_kind == 1) host_minimax_coeffs(n, c->p.eps, cf.data());
        else host_chebyshev_coeffs(n, c->p.eps, cf.data());
        it = c->coeff_sets.emplace(n, std::move(cf)).first;
    }
    return it->second;
}

double delta_of_degree(ov_ctx* c, int n) {
    if (n == c->p.poly_degree) return c->delta;
    auto it = c->delta_of.find(n);
    if (it != c->delta_of.end()) return it->second;
    const std::vector<double>& cf = coeffs_of(c, n);
    const double dl = host_poly_delta(cf.data(), n, c->p.eps);
    c->delta_of[n] = dl;
    return dl;
}

// Smallest degree, a multiple of 8, whose polynomial has delta <= target (delta falls with the
// degree, eq. 2); poly_degree itself when no lower one does or when the coefficients are the
// caller's.
int degree_for_delta(ov_ctx* c, double target) {
    const int N = c->p.poly_degree;
    if (c->custom_coeffs || !(target > c->delta)) return N;
    int lo = 1, hi = (N - 1) / 8;  // degrees 8k < N
    if (hi < 1 || delta_of_degree(c, 8 * hi) > target) return N;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (delta_of_degree(c, 8 * mid) <= target) hi = mid;
        else lo = mid + 1;
    }
    return 8 * lo;
}

// ---- small kernels local to the orchestration --------------------------------

template <typename R>
__global__ void merge_sectors_k(const typename C2<R>::T* __restrict__ Y, const int* __restrict__ sys_of_rhs,
                                typename C2<R>::T* __restrict__ out, long long n) {
    const int j = blockIdx.y;
    const int s0 = sys_of_rhs[2 * j], s1 = sys_of_rhs[2 * j + 1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        typename C2<R>::T v;
        v.x = 0;
        v.y = 0;
        if (s0 >= 0) {
            typename C2<R>::T a = Y[(long long)s0 * n + i];
            v.x += a.x;
            v.y += a.y;
        }
        if (s1 >= 0) {
            typename C2<R>::T a = Y[(long long)s1 * n + i];
            v.x += a.x;
            v.y += a.y;
        }
        out[(long long)j * n + i] = v;
    }
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// x[i] from the numbers of elements i0 + i of the sequence (so that a block filled in pieces gets the
// numbers of one fill)
__global__ void random_fill_k(double2* __restrict__ x, long long n, unsigned long long seed, long long i0) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = (unsigned long long)(i0 + i);
        const unsigned long long a = splitmix64(seed ^ (2ULL * k)), b = splitmix64(seed ^ (2ULL * k + 1));
        x[i] = make_double2((double)(a >> 11) * 0x1.0p-53 - 0.5, (double)(b >> 11) * 0x1.0p-53 - 0.5);
    }
}

// ---- the sign pipeline ---------------------------------------------------------

struct SysSet {
    int n = 0;
    std::vector<double> phase;       // [n]
    std::vector<signed char> chi;    // [n] (may be empty)
};

int upload_sys(ov_ctx* c, const SysSet& S, cudaStream_t s) {
    TRY(ensure_small(c, 0, 0, S.n));
    CK(cudaMemcpyAsync(c->d_phase, S.phase.data(), sizeof(double) * S.n, cudaMemcpyHostToDevice, s));
    if (!S.chi.empty()) CK(cudaMemcpyAsync(c->d_chi, S.chi.data(), S.n, cudaMemcpyHostToDevice, s));
    return OV_OK;
}

bool any_phase(const SysSet& S) {
    for (double p : S.phase)
        if (p != 0.0) return true;
    return false;
}

// Launch shape of the Wilson kernel for ns systems of storage type R (right-hand sides per block;
// for FP32 arithmetic also the 6- or 7-blocks-per-SM register budget and, where the lattice
// allows, the tiled kernel): timed once on the sign pipeline's own buffers (the Clenshaw-step
// launch with its epilogue), fastest kept.
template <typename R>
int tuned_shape(ov_ctx* c, int ns, const void* U, const double* d_phase, void* in, void* v1, void* v2,
                void* v3, void* out, cudaStream_t s) {
    if (c->p.launch_shape > 0) return c->p.launch_shape;  // fixed by the caller
    const auto key = std::make_pair(prec_of<R>(), ns);
    auto it = c->launch_shape.find(key);
    if (it != c->launch_shape.end()) return it->second;
    std::vector<int> shapes;
    for (int by : {1, 2, 4, 8}) {
        if (by > ns) break;
        shapes.push_back(by);
        if (!std::is_same<R, double>::value) {
            shapes.push_back(by | kShapeDense);
            if (tile_rows(c->g, by) > 0) {
                shapes.push_back(by | kShapeTiled);
                shapes.push_back(by | kShapeTiled | kShapeDense);
            }
        }
    }
    int best = shapes[0];
    if (shapes.size() > 1) {
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        Epilogue e;
        e.c_op = 1e-3;
        e.c1 = 1e-3;
        e.v1 = v1;
        e.c2 = 1e-3;
        e.v2 = v2;
        e.c3 = 1e-3;
        e.v3 = v3;
        char buf[64];
        for (int sh : shapes) {
            launch_dslash<R>(c->g, c->p.m0, U, in, out, ns, d_phase, e, s, false, sh);  // warm
            cudaEventRecord(e0, s);
            for (int q = 0; q < 5; ++q) launch_dslash<R>(c->g, c->p.m0, U, in, out, ns, d_phase, e, s, false, sh);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            snprintf(buf, sizeof(buf), "%s%d%s%s:%.1fus", sh == shapes[0] ? "" : " ", sh & kShapeRhsMask,
                     (sh & kShapeDense) ? "d" : "", (sh & kShapeTiled) ? "t" : "", 1e3f * ms / 5);
            c->tune_log += buf;
            if (ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
        }
        c->tune_log += "; ";
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    c->launch_shape[key] = best;
    return best;
}

int take_timeouts() {
    const int a = take_wait_timeouts(), b = take_tc_timeouts();
    if (a < 0 || b < 0) return -1;
    return a | b;
}

// Batches of at least this many FP32 vectors may take the tensor-core projection.
constexpr int kTcMinBatch = 8;

// The small-space projection of k vectors (precision R, internal layout) on the bank b:
// C = V^+ X, Xp = X - V C, Ys = V diag(s) C.  FP32 batches of kTcMinBatch or more vectors go through
// the tcgen05 kernels when the context's method says so, or, by default, when they measured faster for
// this (bank size, batch) the first time it appeared (both paths timed on the call's own buffers).
template <typename R>
int project_bank(ov_ctx* c, const Bank* b, const void* X, int k, void* Xp, void* Ys, cudaStream_t s) {
    const int N = b->n;
    const long long n12 = 12LL * c->g.V;
    const void* Vb = std::is_same<R, double>::value ? b->V64 : b->V32;
    TRY(ensure_small(c, 2LL * N * k, std::max<long long>((long long)N * 4 * 4 * 152, 152LL * N * std::min(k, 32)),
                     std::max(k, 1)));
    int method = 1;
    if (std::is_same<R, float>::value && k >= kTcMinBatch && N <= kTcMaxBank && tc_project_available())
        method = c->proj_method;
    if (method == 1) {
        small_space_project<R>(Vb, N, b->d_signs, X, k, Xp, Ys, n12, c->d_C, c->d_partial, c->partial_cap, s);
        CKL();
        return OV_OK;
    }
    const size_t img = tc_project_image_bytes(N);
    if (c->tc_img.bytes < img) {
        if (c->tc_img.ptr) {
            CK(cudaDeviceSynchronize());
            CK(cudaFree(c->tc_img.ptr));
            c->tc_img.ptr = nullptr;
            c->tc_img.bytes = 0;
        }
        CK(cudaMalloc(&c->tc_img.ptr, img));
        c->tc_img.bytes = img;
    }
    auto run = [&](int m) -> cudaError_t {
        if (m == 2)
            return small_space_project_tc(Vb, N, b->d_signs, X, k, Xp, Ys, n12, c->d_C, c->d_partial, c->partial_cap,
                                          c->tc_img.ptr, s);
        small_space_project<R>(Vb, N, b->d_signs, X, k, Xp, Ys, n12, c->d_C, c->d_partial, c->partial_cap, s);
        return cudaGetLastError();
    };
    if (method == 0) {
        const auto key = std::make_pair(N, k);
        auto it = c->proj_choice.find(key);
        if (it == c->proj_choice.end()) {
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            float ms[3] = {0.f, 0.f, 0.f};
            for (int m : {1, 2}) {
                CK(run(m));  // warm
                CK(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) CK(run(m));
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                CK(cudaEventElapsedTime(&ms[m], e0, e1));
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            const int best = ms[2] < ms[1] ? 2 : 1;
            char buf[128];
            snprintf(buf, sizeof(buf), "projection N %d k %d: cuda cores %.1fus tensor cores %.1fus; ", N, k,
                     1e3f * ms[1] / 3, 1e3f * ms[2] / 3);
            c->tune_log += buf;
            it = c->proj_choice.emplace(key, best).first;
        }
        method = it->second;
    }
    CK(run(method));
    return OV_OK;
}

// out = Proj(G(c_op H_w P(Q^2) x_perp + c1 y_s)) + c2 v2 + c3 v3 over S.n systems of precision R,
// where (y_s, x_perp) is the projection of (g5_in ? gamma5 X : X).  fin.v1 is set here.
// ST: storage of the links and vectors of the recurrence: R itself, or (R = float) a 16-bit
// format, x_perp then being rounded to it and P(Q^2) x_perp read back into FP32 for the final
// FP32 application of H_w.
// degree: of the polynomial (0: the context's poly_degree; lower degrees use the polynomial of
// that degree and the context's kind on the same interval).
template <typename R, typename ST = R>
int sign_pipeline(ov_ctx* c, const void* X, const SysSet& S, bool g5_in, Epilogue fin, void* out, cudaStream_t s,
                  int degree = 0) {
    constexpr bool HALF = !std::is_same<R, ST>::value;
    const int prec = prec_of<R>();
    const int precs = prec_of<ST>();
    const int V = c->g.V;
    const long long n12 = 12LL * V;
    const int ns = S.n;
    TRY(upload_sys(c, S, s));
    const double* d_phase = any_phase(S) ? c->d_phase : nullptr;

    void *xg, *xperp, *ys, *t, *bA, *bB;
    TRY(workspace(c, "sp_xg", prec, ns, &xg));
    TRY(workspace(c, "sp_xperp", prec, ns, &xperp));
    TRY(workspace(c, "sp_ys", prec, ns, &ys));
    TRY(workspace(c, "sp_t", precs, ns, &t));
    TRY(workspace(c, "sp_bA", precs, ns, &bA));
    TRY(workspace(c, "sp_bB", precs, ns, &bB));
    void *xs = xperp, *p32 = nullptr;  // x_perp in the recurrence's storage; FP32 copy of its result
    if (HALF) {
        TRY(workspace(c, "sp_xs", precs, ns, &xs));
        TRY(workspace(c, "sp_p32", prec, ns, &p32));
    }
    const size_t es = sizeof(typename C2<R>::T);

    const void* src = X;
    if (g5_in) {
        launch_gamma5<R>(X, xg, V, ns, s);
        CKL();
        src = xg;
    }

    // small space: runs of equal phase share a bank
    bool any_bank = false;
    for (int j0 = 0; j0 < ns;) {
        int j1 = j0 + 1;
        while (j1 < ns && S.phase[j1] == S.phase[j0]) ++j1;
        const int k = j1 - j0;
        Bank* b = find_bank(c, S.phase[j0]);
        const char* src_j = (const char*)src + (size_t)j0 * n12 * es;
        char* xp_j = (char*)xperp + (size_t)j0 * n12 * es;
        char* ys_j = (char*)ys + (size_t)j0 * n12 * es;
        if (!b && S.phase[j0] != 0.0)
            return fail(c, OV_ERR_NO_BANK, "no small-space bank registered for phase %.17g", S.phase[j0]);
        if (!b || b->n == 0) {
            CK(cudaMemcpyAsync(xp_j, src_j, (size_t)k * n12 * es, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(ys_j, 0, (size_t)k * n12 * es, s));
        } else {
            any_bank = true;
            TRY(ensure_small(c, 0, 0, ns));
            TRY(project_bank<R>(c, b, src_j, k, xp_j, ys_j, s));
        }
        j0 = j1;
    }

    // Clenshaw recurrence for p = P(Q^2) x_perp, P = sum_k c_k T_k(Y),
    // Y = (2 Q^2 - (1 + eps))/(1 - eps) = alpha H_w^2 + beta/2:
    //   b_n = c_n x_perp;  b_k = c_k x_perp + 2 Y b_{k+1} - b_{k+2};
    //   p = c_0 x_perp + Y b_1 - b_2.
    const int n = degree > 0 ? degree : c->p.poly_degree;
    const std::vector<double>& cf = coeffs_of(c, n);
    const double eps = c->p.eps, h = c->hw_norm;
    const double alpha = 4.0 / ((1.0 - eps) * h * h);
    const double beta = -2.0 * (1.0 + eps) / (1.0 - eps);
    const double m0 = c->p.m0;
    const void* U = links_of<R>(c);
    const void* Us = links_of<ST>(c);
    // algorithmic bytes per site of one launch: links once (shared by the systems) plus each
    // system's input, output and epilogue vectors
    const double Vd = (double)V, lb = site_link_bytes(precs), sb = site_spinor_bytes(precs);
    // the whole recurrence (2n launches, no host work) as one stream sequence
    // timing launches read t, bA, x_perp and write bB only (rewritten by the recurrence below)
    const int rb = tuned_shape<ST>(c, ns, Us, d_phase, t, bA, xs, bA, bB, s);
    const int nconv = HALF ? 2 : 1;  // launches before the recurrence
    auto enqueue = [&](cudaStream_t st) -> void* {
        if constexpr (HALF) {
            launch_to_half<ST>(xperp, xs, V, ns, 1.0, st);
            launch_to_half<ST>(xperp, bA, V, ns, cf[n], st);
        } else {
            launch_scale<R>(cf[n], xperp, bA, (long long)ns * n12, st);
        }
        void* b1 = bA;
        void* b2 = nullptr;
        Epilogue plain;
        for (int k = n - 1; k >= 0; --k) {
            launch_dslash<ST>(c->g, m0, Us, b1, t, ns, d_phase, plain, st, false, rb);
            Epilogue e;
            const double half = (k == 0) ? 0.5 : 1.0;
            e.c_op = alpha * half;
            e.c1 = beta * half;
            e.v1 = b1;
            e.c2 = cf[k];
            e.v2 = xs;
            e.c3 = -1.0;
            e.v3 = b2;
            void* o = b2 ? b2 : bB;
            launch_dslash<ST>(c->g, m0, Us, t, o, ns, d_phase, e, st, false, rb);
            b2 = b1;
            b1 = o;
        }
        return b1;
    };
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->profile) {
        CK(cudaEventCreate(&ev0));
        CK(cudaEventCreate(&ev1));
        CK(cudaEventRecord(ev0, s));
        for (int k = n - 1; k >= 0; --k) {
            c->prof_bytes[precs] += Vd * (lb + 2.0 * ns * sb);                          // t = H_w b1
            c->prof_bytes[precs] += Vd * (lb + ns * sb * (k == n - 1 ? 4.0 : 5.0));     // b_k
        }
        c->prof_launches[precs] += 2LL * n;
    }
    void* b1 = nullptr;
    if (c->use_graphs) {
        char key[256];
        snprintf(key, sizeof(key), "%d/%d/%d/%d/%p/%p/%p/%p/%p/%p/%p", precs, n, ns, rb, xperp, xs, bA, bB, t,
                 (const void*)d_phase, Us);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            void* res = enqueue(c->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t e1 = cudaStreamEndCapture(c->cap_stream, &graph);
            if (e1 != cudaSuccess || !graph)
                return fail(c, OV_ERR_CUDA, "graph capture of the polynomial loop failed: %s", cudaGetErrorString(e1));
            cudaGraphExec_t exec = nullptr;
            cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e2 != cudaSuccess) return fail(c, OV_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e2));
            it = c->graphs.emplace(key, std::make_pair(exec, res)).first;
            g_launches.fetch_sub(2LL * n + nconv);  // counted at replay, not at capture
        }
        CK(cudaGraphLaunch(it->second.first, s));
        count_launch(2LL * n + nconv);
        b1 = it->second.second;
    } else {
        b1 = enqueue(s);
    }
    CKL();
    if (c->profile) {
        CK(cudaEventRecord(ev1, s));
        c->prof_events[precs].emplace_back(ev0, ev1);
    }
    // b1 now holds p.  Final: out = Proj(G(c_op H_w p + c1 y_s)) + c2 v2 + c3 v3
    if constexpr (HALF) {
        launch_from_half<ST>(b1, p32, V, ns, s);
        b1 = p32;
    }
    fin.v1 = any_bank ? ys : nullptr;
    launch_dslash<R>(c->g, m0, U, b1, out, ns, d_phase, fin, s);
    CKL();
    c->dslash_count += (long long)(2 * n + 1) * ns;
    c->sign_count += ns;
    return OV_OK;
}

// D(m) X (g5_in = false) or D(m)^+ X (g5_in = true) on internal vectors.
template <typename R, typename ST = R>
int overlap_op(ov_ctx* c, const void* X, const SysSet& S, double mass, bool dagger, void* out, cudaStream_t s,
               int degree = 0) {
    Epilogue fin;
    fin.c_op = (1.0 - 0.5 * mass) / c->hw_norm;
    fin.c1 = 1.0 - 0.5 * mass;
    fin.g5 = dagger ? 0 : 1;
    fin.c2 = 1.0 + 0.5 * mass;
    fin.v2 = X;
    return sign_pipeline<R, ST>(c, X, S, dagger, fin, out, s, degree);
}

// The solver's inner loop runs in FP64, FP32, or with the 16-bit storage of the context's own precision
// (the 16-bit links exist only in an FP16 / BF16 context).
int check_inner_precision(ov_ctx* c, const ov_params* p, int inner) {
    if (inner == OV_PREC_F64 || inner == OV_PREC_F32) return OV_OK;
    if ((inner == OV_PREC_F16 || inner == OV_PREC_BF16) && inner == p->precision) return OV_OK;
    return fail(c, OV_ERR_ARG,
                "inner_precision = %d invalid (FP64, FP32, or the 16-bit format of the context's precision %d)",
                inner, p->precision);
}

int check_ready(ov_ctx* c, const void* in, const void* out, int nrhs) {
    if (!c) return OV_ERR_ARG;
    if (!c->gauge_set) return fail(c, OV_ERR_STATE, "no gauge field set (call ov_set_gauge first)");
    if (!in || !out) return fail(c, OV_ERR_ARG, "null spinor pointer");
    if (in == out) return fail(c, OV_ERR_ARG, "in and out must be different buffers");
    if (nrhs < 1 || nrhs > c->p.max_nrhs)
        return fail(c, OV_ERR_ARG, "nrhs = %d outside [1, max_nrhs = %d]", nrhs, c->p.max_nrhs);
    return OV_OK;
}

SysSet make_sys(int nrhs, const double* phase) {
    SysSet S;
    S.n = nrhs;
    S.phase.assign(nrhs, 0.0);
    if (phase)
        for (int j = 0; j < nrhs; ++j) S.phase[j] = phase[j];
    return S;
}

int phase_check(ov_ctx* c, const SysSet& S) {
    for (double p : S.phase)
        if (!std::isfinite(p)) return fail(c, OV_ERR_ARG, "non-finite phase");
    return OV_OK;
}

// ST: storage of the links and vectors of the Wilson kernels (R, or a 16-bit format with R = float).
template <typename R, typename ST = R>
int apply_generic(ov_ctx* c, const void* in, void* out, int nrhs, const double* phase, int kind, double mass,
                  cudaStream_t s) {
    const int prec = prec_of<R>();
    const int dt = (prec == OV_PREC_F64) ? OV_C128 : OV_C64;
    void *X, *Y;
    TRY(workspace(c, "io_in", prec, nrhs, &X));
    TRY(workspace(c, "io_out", prec, nrhs, &Y));
    launch_pack_spinor<R>(in, dt, X, c->g.V, nrhs, s);
    CKL();
    SysSet S = make_sys(nrhs, phase);
    TRY(phase_check(c, S));
    if (kind == 0 || kind == 1) {  // D_w (0) or H_w (1)
        TRY(upload_sys(c, S, s));
        Epilogue e;
        e.g5 = (kind == 0);  // gamma5 H_w = D_w
        const double* d_phase = any_phase(S) ? c->d_phase : nullptr;
        const int shape = c->p.launch_shape;  // 0: the default shape
        if constexpr (std::is_same<R, ST>::value) {
            launch_dslash<R>(c->g, c->p.m0, links_of<R>(c), X, Y, nrhs, d_phase, e, s, false, shape);
        } else {  // input rounded to the 16-bit format, output read back into FP32
            void *Xh, *Yh;
            TRY(workspace(c, "io_in", prec_of<ST>(), nrhs, &Xh));
            TRY(workspace(c, "io_out", prec_of<ST>(), nrhs, &Yh));
            launch_to_half<ST>(X, Xh, c->g.V, nrhs, 1.0, s);
            launch_dslash<ST>(c->g, c->p.m0, links_of<ST>(c), Xh, Yh, nrhs, d_phase, e, s, false, shape);
            launch_from_half<ST>(Yh, Y, c->g.V, nrhs, s);
        }
        CKL();
        c->dslash_count += nrhs;
    } else if (kind == 2) {  // sign
        Epilogue fin;
        fin.c_op = 1.0 / c->hw_norm;
        fin.c1 = 1.0;
        TRY((sign_pipeline<R, ST>(c, X, S, false, fin, Y, s)));
    } else {  // D(m)
        TRY((overlap_op<R, ST>(c, X, S, mass, false, Y, s)));
    }
    launch_unpack_spinor<R>(Y, out, dt, c->g.V, nrhs, s);
    CKL();
    return OV_OK;
}

int apply_dispatch(ov_ctx* c, const void* in, void* out, int nrhs, const double* phase, int kind, double mass,
                   cudaStream_t s) {
    switch (c->p.precision) {
        case OV_PREC_F64: return apply_generic<double>(c, in, out, nrhs, phase, kind, mass, s);
        case OV_PREC_F32: return apply_generic<float>(c, in, out, nrhs, phase, kind, mass, s);
        case OV_PREC_F16: return apply_generic<float, H16>(c, in, out, nrhs, phase, kind, mass, s);
        default: return apply_generic<float, B16>(c, in, out, nrhs, phase, kind, mass, s);
    }
}

// ---- block helpers for orthonormalisation and Rayleigh-Ritz (FP64) ----------------

// Gram matrix G = W^+ W (m x m) to host, column-major.
template <typename R = double>
int gram_host(ov_ctx* c, const void* A, int na, const void* B, int nb, std::vector<HostCplx>& H, cudaStream_t s) {
    const long long n12 = 12LL * c->g.V;
    TRY(ensure_small(c, (long long)na * nb, (long long)na * nb * 4 * 152, 1));
    multidot<R>(A, n12, na, B, n12, nb, n12, c->d_C, c->d_partial, c->partial_cap, s);
    CKL();
    std::vector<double2> tmp((size_t)na * nb);
    CK(cudaMemcpyAsync(tmp.data(), c->d_C, sizeof(double2) * na * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    H.assign((size_t)na * nb, HostCplx{0, 0});
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) H[i + (size_t)j * na] = HostCplx{tmp[(size_t)i * nb + j].x, tmp[(size_t)i * nb + j].y};
    return OV_OK;
}

// out_j = sum_i A_i M(i, j), M column-major na x nb on the host.
template <typename R = double>
int rotate(ov_ctx* c, const void* A, int na, const std::vector<HostCplx>& M, int nb, void* out, cudaStream_t s) {
    const long long n12 = 12LL * c->g.V;
    TRY(ensure_small(c, (long long)na * nb, 0, 1));
    std::vector<double2> tmp((size_t)na * nb);
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) tmp[(size_t)i * nb + j] = make_double2(M[i + (size_t)j * na].re, M[i + (size_t)j * na].im);
    CK(cudaMemcpyAsync(c->d_C, tmp.data(), sizeof(double2) * na * nb, cudaMemcpyHostToDevice, s));
    combine<R>(A, n12, na, c->d_C, nb, nb, 0.0, nullptr, n12, out, n12, n12, s);
    CKL();
    CK(cudaStreamSynchronize(s));
    return OV_OK;
}

void hermitize(std::vector<HostCplx>& T, int n) {
    for (int i = 0; i < n; ++i) {
        T[i + (size_t)i * n].im = 0.0;
        for (int j = 0; j < i; ++j) {
            HostCplx& x = T[i + (size_t)j * n];
            HostCplx& y = T[j + (size_t)i * n];
            const double re = 0.5 * (x.re + y.re), im = 0.5 * (x.im - y.im);
            x = HostCplx{re, im};
            y = HostCplx{re, -im};
        }
    }
}

// Cholesky-QR, twice: W (m vectors of precision R) <- W R with W^+ W = 1 (Gram and
// triangular factors in FP64 on the host).  tmp: m vectors.
template <typename R = double>
int cholqr2(ov_ctx* c, void* W, int m, void* tmp, cudaStream_t s) {
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<HostCplx> G, Rm;
        TRY(gram_host<R>(c, W, m, W, m, G, s));
        hermitize(G, m);
        if (!host_cholesky(m, G)) return fail(c, OV_ERR_BREAKDOWN, "Cholesky-QR: Gram matrix not positive definite");
        host_inv_lower_dag(m, G, Rm);
        TRY(rotate<R>(c, W, m, Rm, m, tmp, s));
        CK(cudaMemcpyAsync(W, tmp, vec_bytes(c, prec_of<R>()) * m, cudaMemcpyDeviceToDevice, s));
    }
    return OV_OK;
}

int register_bank_internal(ov_ctx* c, double phase, const void* W64, int n, const double* lam, cudaStream_t s) {
    Bank* b = find_bank(c, phase);
    if (!b) {
        c->banks.push_back(Bank());
        b = &c->banks.back();
        b->phase = phase;
    }
    if (b->V64) {
        CK(cudaStreamSynchronize(s));
        CK(cudaFree(b->V64));
        CK(cudaFree(b->V32));
        CK(cudaFree(b->d_signs));
        b->V64 = b->V32 = nullptr;
        b->d_signs = nullptr;
    }
    if (b->Uh64) {
        CK(cudaFree(b->Uh64));
        b->Uh64 = nullptr;
    }
    b->dready = false;
    b->M.clear();
    b->n = n;
    b->signs.assign(n, 1.0);
    b->theta.assign(n, 0.0);
    if (n == 0) return OV_OK;
    for (int i = 0; i < n; ++i) {
        b->signs[i] = (lam[i] >= 0.0) ? 1.0 : -1.0;
        b->theta[i] = lam[i];
    }
    const size_t b64 = vec_bytes(c, OV_PREC_F64) * n, b32 = vec_bytes(c, OV_PREC_F32) * n;
    if (cudaMalloc(&b->V64, b64) != cudaSuccess || cudaMalloc(&b->V32, b32) != cudaSuccess ||
        cudaMalloc(&b->d_signs, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "bank allocation of %d vectors failed", n);
    }
    CK(cudaMemcpy(b->d_signs, b->signs.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpyAsync(b->V64, W64, b64, cudaMemcpyDeviceToDevice, s));
    launch_convert<double, float>(b->V64, b->V32, c->g.V, n, s);
    CKL();
    return OV_OK;
}

// Columns of the eigensolver's block per chunk of its filter and residual passes: three vectors of
// precision prec per column within the context's budget, at least one column.
int eig_chunk(const ov_ctx* c, int prec, int m) {
    const long long per_column = 3LL * (long long)vec_bytes(c, prec);
    return (int)std::max(1LL, std::min<long long>(m, c->eig_chunk_bytes / per_column));
}

// Chebyshev filter W <- T_d(Z) W (then normalised by the caller), Z = (2 Q^2 - (1 + a))/(1 - a),
// which damps the part of the spectrum of Q^2 in [a, 1] and amplifies [0, a).  W: m vectors of
// precision R, filtered a chunk of columns at a time (the recurrence acts on each column alone;
// its three temporaries are chunk-sized).
template <typename R>
int cheb_filter(ov_ctx* c, void* W, int m, double a, int degree, const double* d_phase, cudaStream_t s) {
    const int prec = prec_of<R>();
    const size_t vb = vec_bytes(c, prec);
    const int cw = eig_chunk(c, prec, m);
    void *Tm, *Tc, *tt;
    TRY(workspace(c, "flt_Tm", prec, cw, &Tm));
    TRY(workspace(c, "flt_Tc", prec, cw, &Tc));
    TRY(workspace(c, "flt_t", prec, cw, &tt));
    const double h = c->hw_norm, m0 = c->p.m0;
    const double za = 2.0 / ((1.0 - a) * h * h), zb = -(1.0 + a) / (1.0 - a);
    const void* U = std::is_same<R, double>::value ? c->U64 : c->U32;
    for (int j0 = 0; j0 < m; j0 += cw) {
        const int nj = std::min(cw, m - j0);
        void* Wj = (char*)W + vb * j0;
        Epilogue plain;
        launch_dslash<R>(c->g, m0, U, Wj, tt, nj, d_phase, plain, s);
        Epilogue e1;
        e1.c_op = za;
        e1.c1 = zb;
        e1.v1 = Wj;
        launch_dslash<R>(c->g, m0, U, tt, Tc, nj, d_phase, e1, s);  // T_1 = Z W
        CK(cudaMemcpyAsync(Tm, Wj, vb * nj, cudaMemcpyDeviceToDevice, s));  // T_0
        void* tk = Tc;
        void* tkm = Tm;
        for (int k = 1; k < degree; ++k) {
            launch_dslash<R>(c->g, m0, U, tk, tt, nj, d_phase, plain, s);
            Epilogue e;
            e.c_op = 2.0 * za;
            e.c1 = 2.0 * zb;
            e.v1 = tk;
            e.c3 = -1.0;
            e.v3 = tkm;
            launch_dslash<R>(c->g, m0, U, tt, tkm, nj, d_phase, e, s);  // T_{k+1} written over T_{k-1}
            std::swap(tk, tkm);
        }
        CKL();
        CK(cudaMemcpyAsync(Wj, tk, vb * nj, cudaMemcpyDeviceToDevice, s));
    }
    c->dslash_count += 2LL * degree * m;
    return OV_OK;
}

// Two-stage Rayleigh-Ritz on the block W (m vectors of precision R; Gram matrices and their
// eigenproblems in FP64 on the host).  (1) With Q^2, the operator the filter acts on: orders the
// block by Ritz values of Q^2 and gives the damping bound a.  Ordering by Q instead would pick up
// mixtures of +lambda and -lambda eigenvectors (same Q^2, so the filter never separates them)
// whose Q Rayleigh quotient is near zero.  (2) With Q inside the first n_ev columns: resolves the
// signs; ordered by |theta|.  On return W (and QW) hold the rotated block, theta the Ritz values
// of the first n_ev columns and res their squared residuals ||Q w - theta w||^2.  Three sets of m
// vectors (W, QW and the rotation target W2, whose roles rotate) and a chunk-sized one for the
// residuals.
template <typename R>
int eig_rayleigh_ritz(ov_ctx* c, int m, int n_ev, void*& W, void*& W2, void*& QW, const double* d_phase,
                      std::vector<double>& theta, std::vector<double>& res, double& a, cudaStream_t s) {
    const long long n12 = 12LL * c->g.V;
    const int prec = prec_of<R>();
    const size_t vb = vec_bytes(c, prec);
    const void* U = std::is_same<R, double>::value ? c->U64 : c->U32;
    Epilogue eq;
    eq.c_op = 1.0 / c->hw_norm;
    launch_dslash<R>(c->g, c->p.m0, U, W, QW, m, d_phase, eq, s);
    CKL();
    c->dslash_count += m;
    {
        std::vector<HostCplx> G2, Y;
        std::vector<double> mu;
        TRY(gram_host<R>(c, QW, m, QW, m, G2, s));
        hermitize(G2, m);
        host_eigh(m, G2, mu, Y);
        a = std::min(mu[m - 1], 0.95);
        void* const w_old = W;
        void* const qw_old = QW;
        TRY(rotate<R>(c, W, m, Y, m, W2, s));      // the rotated block
        TRY(rotate<R>(c, QW, m, Y, m, w_old, s));  // its image, over the old block
        W = W2;
        QW = w_old;
        W2 = qw_old;
    }
    std::vector<HostCplx> T, Z;
    TRY(gram_host<R>(c, W, n_ev, QW, n_ev, T, s));
    hermitize(T, n_ev);
    std::vector<double> w;
    host_eigh(n_ev, T, w, Z);
    std::vector<int> order(n_ev);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
        return std::fabs(w[i]) < std::fabs(w[j]) || (std::fabs(w[i]) == std::fabs(w[j]) && w[i] < w[j]);
    });
    std::vector<HostCplx> Zs((size_t)n_ev * n_ev);
    for (int j = 0; j < n_ev; ++j) {
        theta[j] = w[order[j]];
        for (int i = 0; i < n_ev; ++i) Zs[i + (size_t)j * n_ev] = Z[i + (size_t)order[j] * n_ev];
    }
    // rotate the first n_ev columns in place (through W2): the block's span is unchanged
    TRY(rotate<R>(c, W, n_ev, Zs, n_ev, W2, s));
    CK(cudaMemcpyAsync(W, W2, vb * n_ev, cudaMemcpyDeviceToDevice, s));
    TRY(rotate<R>(c, QW, n_ev, Zs, n_ev, W2, s));
    CK(cudaMemcpyAsync(QW, W2, vb * n_ev, cudaMemcpyDeviceToDevice, s));
    std::vector<double> mth(n_ev), ones(n_ev, 1.0);
    for (int i = 0; i < n_ev; ++i) mth[i] = -theta[i];
    const int cw = eig_chunk(c, prec, n_ev);
    void* tt;
    TRY(workspace(c, "eig_t", prec, cw, &tt));
    TRY(ensure_small(c, 0, (long long)kRedBlocks * cw, cw));
    for (int j0 = 0; j0 < n_ev; j0 += cw) {
        const int nj = std::min(cw, n_ev - j0);
        CK(cudaMemcpyAsync(tt, (const char*)QW + vb * j0, vb * nj, cudaMemcpyDeviceToDevice, s));
        launch_axpby<R>(mth.data() + j0, (const char*)W + vb * j0, ones.data() + j0, tt, n12, nj, s);
        CKL();
        norm2_rhs<R>(tt, n12, nj, res.data() + j0, c->d_partial, c->d_red, s);
    }
    return OV_OK;
}

}  // namespace

void ovl::set_global_error(const char* msg) { g_create_error = msg; }

// ============================================================================
// C ABI
// ============================================================================

extern "C" {

int ov_create(const ov_params* p, ov_ctx** out) {
    ov_ctx* c = nullptr;
    if (!p || !out) return fail(c, OV_ERR_ARG, "null argument");
    *out = nullptr;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (p->dims[mu] < 2) return fail(c, OV_ERR_ARG, "dims[%d] = %d < 2", mu, p->dims[mu]);
        if (p->bc[mu] < 0 || p->bc[mu] > 2) return fail(c, OV_ERR_ARG, "bc[%d] = %d invalid", mu, p->bc[mu]);
        // checked before each product (V <= 2^30 / 12 and an int extent cannot overflow 64 bits)
        V *= p->dims[mu];
        if (V > (1LL << 30) / 12) return fail(c, OV_ERR_ARG, "lattice too large for 32-bit site indexing");
    }
    if (!(p->eps > 0.0 && p->eps < 1.0)) return fail(c, OV_ERR_ARG, "eps = %g outside (0, 1)", p->eps);
    if (p->poly_degree < 1 || p->poly_degree > 100000)
        return fail(c, OV_ERR_ARG, "poly_degree = %d outside [1, 100000]", p->poly_degree);
    if (p->precision < OV_PREC_F64 || p->precision > OV_PREC_BF16)
        return fail(c, OV_ERR_ARG, "precision = %d invalid", p->precision);
    TRY(check_inner_precision(c, p, p->inner_precision));
    if (p->max_nrhs < 1 || p->max_nrhs > kMaxRhs / 2)
        return fail(c, OV_ERR_ARG, "max_nrhs = %d outside [1, %d]", p->max_nrhs, kMaxRhs / 2);
    if (!std::isfinite(p->m0)) return fail(c, OV_ERR_ARG, "m0 not finite");
    if (p->poly_kind != 0 && p->poly_kind != 1) return fail(c, OV_ERR_ARG, "poly_kind = %d invalid", p->poly_kind);
    if (p->poly_kind == 1 && p->poly_degree > 4000)
        return fail(c, OV_ERR_ARG, "poly_degree = %d above 4000 for the minimax polynomial", p->poly_degree);
    {
        const int rb = p->launch_shape & kShapeRhsMask;
        if (p->launch_shape < 0 || (p->launch_shape & ~(kShapeRhsMask | kShapeDense | kShapeTiled)) ||
            (p->launch_shape > 0 && rb != 1 && rb != 2 && rb != 4 && rb != 8))
            return fail(c, OV_ERR_ARG, "launch_shape = %d invalid", p->launch_shape);
    }
    c = new ov_ctx();
    c->p = *p;
    for (int mu = 0; mu < 4; ++mu) {
        c->g.L[mu] = p->dims[mu];
        c->g.bcf[mu] = p->bc[mu] == OV_BC_PERIODIC ? 1.0 : (p->bc[mu] == OV_BC_ANTIPERIODIC ? -1.0 : 0.0);
    }
    c->g.V = (int)V;
    c->coeffs.resize(p->poly_degree + 1);
    if (p->coeffs) std::copy(p->coeffs, p->coeffs + p->poly_degree + 1, c->coeffs.begin());
    else if (p->poly_kind == 1) host_minimax_coeffs(p->poly_degree, p->eps, c->coeffs.data());
    else host_chebyshev_coeffs(p->poly_degree, p->eps, c->coeffs.data());
    c->p.coeffs = nullptr;
    c->hw_norm = p->hw_norm > 0.0 ? p->hw_norm : std::fabs(4.0 + p->m0) + 4.0;
    c->delta = host_poly_delta(c->coeffs.data(), p->poly_degree, p->eps);
    c->custom_coeffs = p->coeffs != nullptr;
    if (c->p.max_iter <= 0) c->p.max_iter = 100000;
    *out = c;
    return OV_OK;
}

int ov_destroy(ov_ctx* c) {
    if (!c) return OV_OK;
    cudaDeviceSynchronize();
    for (auto& kv : c->ws)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    for (auto& b : c->banks) {
        if (b.V64) cudaFree(b.V64);
        if (b.V32) cudaFree(b.V32);
        if (b.d_signs) cudaFree(b.d_signs);
        if (b.Uh64) cudaFree(b.Uh64);
    }
    for (auto& sp : c->dspaces)
        for (void* q : {sp.W, sp.AW0, sp.AWm, sp.W64, sp.DW64, sp.DmW64, sp.AW64, sp.AWm64})
            if (q) cudaFree(q);
    if (c->tc_img.ptr) cudaFree(c->tc_img.ptr);
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto& v : c->prof_events)
        for (auto& e : v) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    void* ps[] = {c->U64, c->U32, c->U16, c->d_partial, c->d_red, c->d_C, c->d_C2, c->d_phase, c->d_chi, c->d_idx};
    for (void* q : ps)
        if (q) cudaFree(q);
    delete c;
    return OV_OK;
}

const char* ov_last_error(const ov_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char* ov_last_info(const ov_ctx* c) { return c ? c->info.c_str() : ""; }

const char* ov_tune_info(const ov_ctx* c) { return c ? c->tune_log.c_str() : ""; }

int ov_selftest_bounded_wait(ov_ctx* c, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    launch_bounded_wait_selftest(2000000LL, (cudaStream_t)stream);  // about a millisecond
    CKL();
    return OV_OK;
}

int ov_sync(ov_ctx* c, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    const int t = take_timeouts();
    if (t < 0) return fail(c, OV_ERR_CUDA, "reading the device wait flag failed");
    if (t > 0) return fail(c, OV_ERR_TIMEOUT, "a bounded device wait ran out");
    return OV_OK;
}

long long ov_volume(const ov_ctx* c) { return c ? c->g.V : 0; }

double ov_hw_norm(const ov_ctx* c) { return c ? c->hw_norm : 0.0; }

double ov_poly_delta(const ov_ctx* c) { return c ? c->delta : 0.0; }

double ov_poly_delta_n(int n, double eps) {
    if (n < 1 || n > 100000 || !(eps > 0.0 && eps < 1.0)) return -1.0;
    std::vector<double> cf(n + 1);
    host_chebyshev_coeffs(n, eps, cf.data());
    return host_poly_delta(cf.data(), n, eps);
}

double ov_minimax_coeffs(int n, double eps, double* out) {
    if (n < 0 || n > 4000 || !out || !(eps > 0.0 && eps < 1.0)) return -1.0;
    return host_minimax_coeffs(n, eps, out);
}

int ov_adaptive_degree(ov_ctx* c, double delta_target) {
    if (!c) return 0;
    return degree_for_delta(c, delta_target);
}

int ov_chebyshev_coeffs(int n, double eps, double* out) {
    if (n < 0 || !out || !(eps > 0.0 && eps < 1.0)) return OV_ERR_ARG;
    host_chebyshev_coeffs(n, eps, out);
    return OV_OK;
}

int ov_host_eigh(int n, double* A, double* w, double* Z) {
    if (n < 1 || !A || !w || !Z) return OV_ERR_ARG;
    std::vector<HostCplx> M((size_t)n * n), Zm;
    std::memcpy(M.data(), A, sizeof(HostCplx) * n * n);
    std::vector<double> wv;
    host_eigh(n, M, wv, Zm);
    std::memcpy(w, wv.data(), sizeof(double) * n);
    std::memcpy(Z, Zm.data(), sizeof(HostCplx) * n * n);
    return OV_OK;
}

int ov_set_profiling(ov_ctx* c, int on) {
    if (!c) return OV_ERR_ARG;
    c->profile = on != 0;
    return OV_OK;
}

int ov_read_profile(ov_ctx* c, int precision, ov_profile* out) {
    if (!c || !out || precision < OV_PREC_F64 || precision > OV_PREC_BF16) return OV_ERR_ARG;
    const int p = precision;
    double ms = 0.0;
    for (auto& e : c->prof_events[p]) {
        CK(cudaEventSynchronize(e.second));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e.first, e.second));
        ms += t;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    out->clenshaw_ms = ms;
    out->clenshaw_regions = (long long)c->prof_events[p].size();
    out->clenshaw_launches = c->prof_launches[p];
    out->clenshaw_bytes = c->prof_bytes[p];
    out->kernel_launches = g_launches.load();
    c->prof_events[p].clear();
    c->prof_launches[p] = 0;
    c->prof_bytes[p] = 0.0;
    return OV_OK;
}

long long ov_launch_count(void) { return g_launches.load(); }

int ov_set_gauge(ov_ctx* c, const void* U, int dtype, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    if (!U) return fail(c, OV_ERR_ARG, "null gauge pointer");
    if (dtype != OV_C128 && dtype != OV_C64) return fail(c, OV_ERR_ARG, "dtype = %d invalid", dtype);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = 4ull * 9 * c->g.V;
    const bool half = c->p.precision == OV_PREC_F16 || c->p.precision == OV_PREC_BF16;
    if (!c->U64) {
        if (cudaMalloc(&c->U64, n * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&c->U32, 4ull * 3 * c->g.V * sizeof(float4)) != cudaSuccess ||
            (half && cudaMalloc(&c->U16, 96ull * c->g.V) != cudaSuccess)) {
            cudaGetLastError();
            return fail(c, OV_ERR_OOM, "gauge field allocation failed");
        }
    }
    launch_pack_gauge<double>(U, dtype, c->U64, c->g, s);
    launch_pack_gauge<float>(U, dtype, c->U32, c->g, s);
    if (c->p.precision == OV_PREC_F16) launch_pack_gauge_half<H16>(U, dtype, c->U16, c->g.V, s);
    if (c->p.precision == OV_PREC_BF16) launch_pack_gauge_half<B16>(U, dtype, c->U16, c->g.V, s);
    CKL();
    c->gauge_set = true;
    return OV_OK;
}

int apply_wilson(ov_ctx* c, const void* in, void* out, int nrhs, const double* phase, int hermitian,
                 ov_stream_t stream) {
    TRY(check_ready(c, in, out, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    return apply_dispatch(c, in, out, nrhs, phase, hermitian ? 1 : 0, 0.0, s);
}

int apply_sign_Hw(ov_ctx* c, const void* in, void* out, int nrhs, const double* phase, ov_stream_t stream) {
    TRY(check_ready(c, in, out, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    return apply_dispatch(c, in, out, nrhs, phase, 2, 0.0, s);
}

int apply_overlap(ov_ctx* c, const void* in, void* out, int nrhs, double mass, const double* phase,
                  ov_stream_t stream) {
    TRY(check_ready(c, in, out, nrhs));
    if (!std::isfinite(mass)) return fail(c, OV_ERR_ARG, "mass not finite");
    cudaStream_t s = (cudaStream_t)stream;
    return apply_dispatch(c, in, out, nrhs, phase, 3, mass, s);
}

int ov_set_projection(ov_ctx* c, int method) {
    if (!c) return OV_ERR_ARG;
    if (method < 0 || method > 2) return fail(c, OV_ERR_ARG, "projection method = %d invalid", method);
    if (method == 2 && !tc_project_available())
        return fail(c, OV_ERR_ARG, "tensor-core projection unavailable (no tensor-map encoder in the driver)");
    c->proj_method = method;
    return OV_OK;
}

int ov_set_eigensolver_memory(ov_ctx* c, long long bytes) {
    if (!c) return OV_ERR_ARG;
    if (bytes < 1) return fail(c, OV_ERR_ARG, "eigensolver memory budget = %lld bytes invalid", bytes);
    c->eig_chunk_bytes = bytes;
    return OV_OK;
}

int ov_project_small(ov_ctx* c, double phase, const void* in, void* ys, void* xperp, int nrhs, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    if (!in || !ys || !xperp) return fail(c, OV_ERR_ARG, "null spinor pointer");
    if (in == ys || in == xperp || ys == xperp) return fail(c, OV_ERR_ARG, "in, ys and xperp must be different buffers");
    if (nrhs < 1 || nrhs > c->p.max_nrhs)
        return fail(c, OV_ERR_ARG, "nrhs = %d outside [1, max_nrhs = %d]", nrhs, c->p.max_nrhs);
    if (!std::isfinite(phase)) return fail(c, OV_ERR_ARG, "non-finite phase");
    Bank* b = find_bank(c, phase);
    if (!b && phase != 0.0) return fail(c, OV_ERR_NO_BANK, "no small-space bank registered for phase %.17g", phase);
    cudaStream_t s = (cudaStream_t)stream;
    const bool f64 = c->p.precision == OV_PREC_F64;
    const int prec = f64 ? OV_PREC_F64 : OV_PREC_F32, dt = f64 ? OV_C128 : OV_C64;
    void *X, *P, *Y;
    TRY(workspace(c, "pj_in", prec, nrhs, &X));
    TRY(workspace(c, "pj_xp", prec, nrhs, &P));
    TRY(workspace(c, "pj_ys", prec, nrhs, &Y));
    const size_t bytes = vec_bytes(c, prec) * nrhs;
    if (f64) launch_pack_spinor<double>(in, dt, X, c->g.V, nrhs, s);
    else launch_pack_spinor<float>(in, dt, X, c->g.V, nrhs, s);
    CKL();
    if (!b || b->n == 0) {
        CK(cudaMemcpyAsync(P, X, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(Y, 0, bytes, s));
    } else if (f64) {
        TRY(project_bank<double>(c, b, X, nrhs, P, Y, s));
    } else {
        TRY(project_bank<float>(c, b, X, nrhs, P, Y, s));
    }
    if (f64) {
        launch_unpack_spinor<double>(P, xperp, dt, c->g.V, nrhs, s);
        launch_unpack_spinor<double>(Y, ys, dt, c->g.V, nrhs, s);
    } else {
        launch_unpack_spinor<float>(P, xperp, dt, c->g.V, nrhs, s);
        launch_unpack_spinor<float>(Y, ys, dt, c->g.V, nrhs, s);
    }
    CKL();
    return OV_OK;
}

int deflate(ov_ctx* c, double phase, const void* V, const double* lambda, int n_ev, int dtype, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_ev < 0 || n_ev > 384) return fail(c, OV_ERR_ARG, "n_ev = %d outside [0, 384]", n_ev);
    if (n_ev > 0 && (!V || !lambda)) return fail(c, OV_ERR_ARG, "null V or lambda");
    if (dtype != OV_C128 && dtype != OV_C64) return fail(c, OV_ERR_ARG, "dtype = %d invalid", dtype);
    if (!std::isfinite(phase)) return fail(c, OV_ERR_ARG, "non-finite phase");
    if (n_ev == 0) return register_bank_internal(c, phase, nullptr, 0, nullptr, s);
    for (int i = 0; i < n_ev; ++i)
        if (!std::isfinite(lambda[i])) return fail(c, OV_ERR_ARG, "lambda[%d] not finite", i);
    void *W, *T;
    TRY(workspace(c, "defl_W", OV_PREC_F64, n_ev, &W));
    TRY(workspace(c, "defl_T", OV_PREC_F64, n_ev, &T));
    launch_pack_spinor<double>(V, dtype, W, c->g.V, n_ev, s);
    CKL();
    TRY(cholqr2(c, W, n_ev, T, s));
    return register_bank_internal(c, phase, W, n_ev, lambda, s);
}

static int eigensolve_q_body(ov_ctx* c, double phase, int n_ev, double tol, int max_iter, void* V_out,
                             double* lambda_out, int register_bank, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    if (!c->gauge_set) return fail(c, OV_ERR_STATE, "no gauge field set");
    if (n_ev < 1 || n_ev > 200) return fail(c, OV_ERR_ARG, "n_ev = %d outside [1, 200]", n_ev);
    if (!lambda_out) return fail(c, OV_ERR_ARG, "null lambda_out");
    if (!(tol > 0.0)) return fail(c, OV_ERR_ARG, "tol must be > 0");
    if (!std::isfinite(phase)) return fail(c, OV_ERR_ARG, "non-finite phase");
    cudaStream_t s = (cudaStream_t)stream;
    // block = wanted + guard; a deep guard puts the damping edge a beyond the cluster the
    // wanted set ends in (near-degenerate modes at the cut converge at the rate set by a)
    const int m = std::min(std::min(n_ev + std::max(16, n_ev), 12 * c->g.V), kMaxRhs);
    const long long n12 = 12LL * c->g.V;
    const size_t vb32 = vec_bytes(c, OV_PREC_F32);
    // the block lives in FP32 while the residuals are well above FP32 resolution (filter,
    // Cholesky-QR and Rayleigh-Ritz all on FP32 vectors), then in FP64.
    // Memory: three sets of m vectors (block, image under Q, rotation target) in FP32 until the
    // switch to FP64 and in FP64 after it, chunk-sized sets for the filter and the residuals, and at
    // the end the n_ev wanted vectors in FP64; all released when the call returns.
    void *W = nullptr, *W2 = nullptr, *QW = nullptr, *Wf, *W2f, *QWf;
    TRY(workspace(c, "eig_W", OV_PREC_F32, m, &Wf));
    TRY(workspace(c, "eig_W2", OV_PREC_F32, m, &W2f));
    TRY(workspace(c, "eig_QW", OV_PREC_F32, m, &QWf));
    {  // random start block, drawn in FP64 a chunk of columns at a time
        const int cw = eig_chunk(c, OV_PREC_F64, m);
        void* r64;
        TRY(workspace(c, "eig_r", OV_PREC_F64, cw, &r64));
        for (int j0 = 0; j0 < m; j0 += cw) {
            const int nj = std::min(cw, m - j0);
            random_fill_k<<<152 * 8, 256, 0, s>>>((double2*)r64, n12 * nj, 0x5eed0f0e1ULL, n12 * j0);
            count_launch();
            launch_convert<double, float>(r64, (char*)Wf + vb32 * j0, c->g.V, nj, s);
        }
        CKL();
        TRY(release_workspaces(c, "eig_r/", s));
    }
    // warm start: the bank of the nearest other field phase, if one is registered, replaces the first
    // random vectors (the field moves the low modes of Q little at the phases of the background-field
    // method, so the filter then only has to correct them); its FP32 copy is its FP64 vectors rounded
    const Bank* warm = nullptr;
    for (const Bank& bk : c->banks)
        if (bk.n > 0 && bk.phase != phase && (!warm || std::fabs(bk.phase - phase) < std::fabs(warm->phase - phase)))
            warm = &bk;
    if (warm) CK(cudaMemcpyAsync(Wf, warm->V32, vb32 * std::min(warm->n, m), cudaMemcpyDeviceToDevice, s));
    TRY(cholqr2<float>(c, Wf, m, W2f, s));
    SysSet S;
    S.n = m;
    S.phase.assign(m, phase);
    TRY(upload_sys(c, S, s));
    const double* d_phase = phase != 0.0 ? c->d_phase : nullptr;
    // The filter degree is chosen each cycle so that the largest amplification, |T_d(z(0))|
    // with z(0) = -(1 + a)/(1 - a), stays below amp: a larger spread between the filtered
    // columns would collapse the block below the resolution of the Cholesky-QR step.
    // FP32 resolves residuals down to a few 1e-7: a target of 2e-6 or more is met without the FP64 phase
    const double switch_res = tol >= 2e-6 ? 0.0 : 3e-6;
    double prev_worst = 1e300;
    bool in_f64 = false;
    double a = -1.0;  // lower end of the damped interval of Q^2 (set by each Rayleigh-Ritz)
    std::vector<double> theta(m), res(m, 1e300);
    double worst = 1e300;
    int status = OV_ERR_NOT_CONVERGED;
    std::string hist;
    double t_filter[2] = {0.0, 0.0}, t_ortho = 0.0, t_rr = 0.0;
    const auto t_start = std::chrono::steady_clock::now();
    auto since = [](std::chrono::steady_clock::time_point t0) {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    for (int it = 0; it <= max_iter; ++it) {
        int degree = 0;
        if (it > 0) {
            if (!in_f64 && (worst <= switch_res || (switch_res > 0.0 && worst < 1e-4 && worst > 0.9 * prev_worst))) {
                // FP32 -> FP64: widen the block and restore FP64 orthonormality
                TRY(workspace(c, "eig_W", OV_PREC_F64, m, &W));
                launch_convert<float, double>(Wf, W, c->g.V, m, s);
                CKL();
                TRY(release_workspaces(c, "flt_", s));
                for (const char* nm : {"eig_W/32", "eig_W2/32", "eig_QW/32", "eig_t/32"}) TRY(release_workspaces(c, nm, s));
                TRY(workspace(c, "eig_W2", OV_PREC_F64, m, &W2));
                TRY(workspace(c, "eig_QW", OV_PREC_F64, m, &QW));
                auto t0 = std::chrono::steady_clock::now();
                TRY(cholqr2<double>(c, W, m, W2, s));
                t_ortho += since(t0);
                in_f64 = true;
            }
            prev_worst = worst;
            const double amp = in_f64 ? 1e6 : 1e3;
            const double z0 = (1.0 + a) / (1.0 - a);
            degree = std::max(2, std::min(200, (int)std::ceil(std::acosh(amp) / std::acosh(z0))));
            auto tf = std::chrono::steady_clock::now();
            if (in_f64) TRY(cheb_filter<double>(c, W, m, a, degree, d_phase, s));
            else TRY(cheb_filter<float>(c, Wf, m, a, degree, d_phase, s));
            CK(cudaStreamSynchronize(s));
            auto to = std::chrono::steady_clock::now();
            t_filter[in_f64 ? 1 : 0] += std::chrono::duration<double>(to - tf).count();
            if (in_f64) TRY(cholqr2<double>(c, W, m, W2, s));
            else TRY(cholqr2<float>(c, Wf, m, W2f, s));
            t_ortho += since(to);
        }
        const auto t_rr0 = std::chrono::steady_clock::now();
        if (in_f64) TRY(eig_rayleigh_ritz<double>(c, m, n_ev, W, W2, QW, d_phase, theta, res, a, s));
        else TRY(eig_rayleigh_ritz<float>(c, m, n_ev, Wf, W2f, QWf, d_phase, theta, res, a, s));
        t_rr += since(t_rr0);
        worst = 0.0;
        for (int i = 0; i < n_ev; ++i) worst = std::max(worst, std::sqrt(res[i]));
        char buf[96];
        snprintf(buf, sizeof(buf), "%s%s%d:%.1e", it ? " " : "", it == 0 ? "" : (in_f64 ? "f64/" : "f32/"), degree,
                 worst);
        hist += buf;
        if (worst <= tol) {
            status = OV_OK;
            break;
        }
    }
    if (!in_f64) {  // converged (or stopped) in FP32: hand out the n_ev wanted vectors in FP64,
                    // orthonormalised in FP64 (the first n_ev columns of a Cholesky-QR of the block)
        TRY(release_workspaces(c, "flt_", s));
        TRY(release_workspaces(c, "eig_t/32", s));
        TRY(workspace(c, "eig_W", OV_PREC_F64, n_ev, &W));
        launch_convert<float, double>(Wf, W, c->g.V, n_ev, s);
        CKL();
        for (const char* nm : {"eig_W/32", "eig_W2/32", "eig_QW/32"}) TRY(release_workspaces(c, nm, s));
        TRY(workspace(c, "eig_W2", OV_PREC_F64, n_ev, &W2));
        TRY(cholqr2<double>(c, W, n_ev, W2, s));
        TRY(release_workspaces(c, "eig_W2/64", s));
    }
    for (int i = 0; i < n_ev; ++i) lambda_out[i] = theta[i];
    if (V_out) {
        launch_unpack_spinor<double>(W, V_out, OV_C128, c->g.V, n_ev, s);
        CKL();
    }
    if (register_bank && status == OV_OK) TRY(register_bank_internal(c, phase, W, n_ev, theta.data(), s));
    CK(cudaStreamSynchronize(s));
    // the block's workspaces are the largest the library holds; they serve only this call
    TRY(release_workspaces(c, "eig_", s));
    TRY(release_workspaces(c, "flt_", s));
    if (take_timeouts() > 0) return fail(c, OV_ERR_TIMEOUT, "eigensolver: a bounded device wait ran out");
    {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "eigensolver: n_ev %d, block %d%s, %.1f s (filter f32 %.1f, f64 %.1f, orthonormalise %.1f, "
                 "Rayleigh-Ritz %.1f); per cycle [precision/degree:]worst residual: ",
                 n_ev, m, warm ? " (warm start from another phase's bank)" : "", since(t_start), t_filter[0],
                 t_filter[1], t_ortho, t_rr);
        c->info = std::string(buf) + hist;
    }
    if (status != OV_OK)
        return fail(c, status, "eigensolver: not converged after %d filter cycles; worst residual per cycle: %s",
                    max_iter, hist.c_str());
    return OV_OK;
}

int ov_eigensolve_Q(ov_ctx* c, double phase, int n_ev, double tol, int max_iter, void* V_out, double* lambda_out,
                    int register_bank, ov_stream_t stream) {
    const int rc = eigensolve_q_body(c, phase, n_ev, tol, max_iter, V_out, lambda_out, register_bank, stream);
    // a call that failed part-way (out of memory, a CUDA error) gives its block back as well
    if (c && rc != OV_OK && rc != OV_ERR_NOT_CONVERGED) {
        release_workspaces_after_error(c, "eig_", (cudaStream_t)stream);
        release_workspaces_after_error(c, "flt_", (cudaStream_t)stream);
    }
    return rc;
}

}  // extern "C"

// ---- solver ----------------------------------------------------------------------

namespace {

// ---- D_ov low modes and the deflated inner CG (Sec. 3.2) ----------------------------

DefSpace* find_dspace(ov_ctx* c, double phase, int chi) {
    for (auto& sp : c->dspaces)
        if (sp.phase == phase && sp.chi == chi && sp.n > 0) return &sp;
    return nullptr;
}

// Epilogue of the chiral-sector operator A(m) = P_s [k1 (1 + s sign) + m^2] P_s, k1 = 2 (1 - m^2/4),
// applied to v (one sign application per system; the systems' chiralities in c->d_chi).
Epilogue sector_operator(const ov_ctx* c, double mass, const void* v) {
    const double k1 = 2.0 * (1.0 - 0.25 * mass * mass);
    Epilogue fin;
    fin.c_op = k1 / c->hw_norm;
    fin.c1 = k1;
    fin.chi = c->d_chi;
    fin.c2 = k1 + mass * mass;
    fin.v2 = v;
    return fin;
}

int dspace_prepare_dm(ov_ctx* c, DefSpace& sp, double mass, cudaStream_t s);

// Inverse of a Hermitian positive-definite matrix (column-major n x n; hermitised first).
bool hpd_inverse(std::vector<HostCplx> E, int n, std::vector<HostCplx>& out) {
    hermitize(E, n);
    if (!host_cholesky(n, E)) return false;
    std::vector<HostCplx> Rm;
    host_inv_lower_dag(n, E, Rm);  // Rm = L^{-+}, E^{-1} = Rm Rm^+
    out.assign((size_t)n * n, HostCplx{0, 0});
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < n; ++k) {
                const HostCplx x = Rm[i + (size_t)k * n], y = Rm[j + (size_t)k * n];  // x * conj(y)
                re += x.re * y.re + x.im * y.im;
                im += x.im * y.re - x.re * y.im;
            }
            out[i + (size_t)j * n] = HostCplx{re, im};
        }
    return true;
}

// A(m) W = (1 - m^2/4) A0 W + m^2 W and (W^+ A(m) W)^{-1} for this mass (kept until the mass changes).
int dspace_prepare(ov_ctx* c, DefSpace& sp, double mass, cudaStream_t s) {
    if (sp.mass == mass && sp.AWm) return OV_OK;
    const int n = sp.n;
    const long long n12 = 12LL * c->g.V;
    if (!sp.AWm && cudaMalloc(&sp.AWm, vec_bytes(c, OV_PREC_F32) * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "deflation space: allocation of %d vectors failed", n);
    }
    std::vector<double> a(n, 1.0 - 0.25 * mass * mass), m2(n, mass * mass);
    CK(cudaMemcpyAsync(sp.AWm, sp.W, vec_bytes(c, OV_PREC_F32) * n, cudaMemcpyDeviceToDevice, s));
    launch_axpby<float>(a.data(), sp.AW0, m2.data(), sp.AWm, n12, n, s);
    CKL();
    std::vector<HostCplx> E;
    TRY(gram_host<float>(c, sp.W, n, sp.AWm, n, E, s));
    if (!hpd_inverse(E, n, sp.Einv)) return fail(c, OV_ERR_BREAKDOWN, "deflation space: W^+ A W not positive definite");
    sp.mass = mass;
    return OV_OK;
}

// The FP64 counterparts for this mass: A(m) W = (1 - m^2/4) A0 W + m^2 W and (W^+ A(m) W)^{-1}.
int dspace_prepare64(ov_ctx* c, DefSpace& sp, double mass, cudaStream_t s) {
    if (sp.AWm64 && sp.dm_mass == mass && !sp.Einv64.empty()) return OV_OK;
    const int n = sp.n;
    const size_t b64 = vec_bytes(c, OV_PREC_F64) * n;
    if (!sp.AWm64 && cudaMalloc(&sp.AWm64, b64) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "deflation space: allocation of %d FP64 vectors failed", n);
    }
    std::vector<double> a(n, 1.0 - 0.25 * mass * mass), m2(n, mass * mass);
    CK(cudaMemcpyAsync(sp.AWm64, sp.W64, b64, cudaMemcpyDeviceToDevice, s));
    launch_axpby<double>(a.data(), sp.AW64, m2.data(), sp.AWm64, 12LL * c->g.V, n, s);
    CKL();
    std::vector<HostCplx> E;
    TRY(gram_host<double>(c, sp.W64, n, sp.AWm64, n, E, s));
    if (!hpd_inverse(E, n, sp.Einv64))
        return fail(c, OV_ERR_BREAKDOWN, "deflation space: W^+ A W (FP64) not positive definite");
    TRY(dspace_prepare_dm(c, sp, mass, s));  // sets dm_mass
    return OV_OK;
}

// out (host, n) = Einv * (A_i^+ v for the n vectors A of the space), A = AWm or W, in precision R
// (FP32: the FP32 vectors and Einv; FP64: the FP64 vectors and Einv64).
template <typename R = float>
int dspace_coeffs(ov_ctx* c, DefSpace& sp, const void* A, const void* v, std::vector<HostCplx>& out, bool apply_einv,
                  cudaStream_t s) {
    std::vector<HostCplx> g;
    TRY(gram_host<R>(c, A, sp.n, v, 1, g, s));
    const std::vector<HostCplx>& Einv = std::is_same<R, double>::value ? sp.Einv64 : sp.Einv;
    if (!apply_einv) {
        out = g;
        return OV_OK;
    }
    const int n = sp.n;
    out.assign(n, HostCplx{0, 0});
    for (int i = 0; i < n; ++i) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < n; ++k) {
            const HostCplx e = Einv[i + (size_t)k * n], x = g[k];
            re += e.re * x.re - e.im * x.im;
            im += e.re * x.im + e.im * x.re;
        }
        out[i] = HostCplx{re, im};
    }
    return OV_OK;
}

// out = X + sign * sum_i A_i coef_i (one vector of precision R; out must not alias X).
template <typename R = float>
int dspace_combine(ov_ctx* c, const void* A, int n, const std::vector<HostCplx>& coef, double sign, const void* X,
                   void* out, cudaStream_t s) {
    std::vector<HostCplx> M(n);
    for (int i = 0; i < n; ++i) M[i] = HostCplx{sign * coef[i].re, sign * coef[i].im};
    const long long n12 = 12LL * c->g.V;
    TRY(ensure_small(c, n, 0, 1));
    std::vector<double2> tmp(n);
    for (int i = 0; i < n; ++i) tmp[i] = make_double2(M[i].re, M[i].im);
    CK(cudaMemcpyAsync(c->d_C, tmp.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, s));
    combine<R>(A, n12, n, c->d_C, 1, 1, X ? 1.0 : 0.0, X, n12, out, n12, n12, s);
    CKL();
    return OV_OK;
}

// D(m)^+ W = (1 - m/2) D_ov^+ W + m W in FP64 for this mass.
int dspace_prepare_dm(ov_ctx* c, DefSpace& sp, double mass, cudaStream_t s) {
    if (!sp.DW64) return OV_OK;
    if (sp.dm_mass == mass && sp.DmW64) return OV_OK;
    const size_t b64 = vec_bytes(c, OV_PREC_F64) * sp.n;
    if (!sp.DmW64 && cudaMalloc(&sp.DmW64, b64) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "deflation space: allocation of %d FP64 vectors failed", sp.n);
    }
    std::vector<double> a(sp.n, 1.0 - 0.5 * mass), mm(sp.n, mass);
    CK(cudaMemcpyAsync(sp.DmW64, sp.W64, b64, cudaMemcpyDeviceToDevice, s));
    launch_axpby<double>(a.data(), sp.DW64, mm.data(), sp.DmW64, 12LL * c->g.V, sp.n, s);
    CKL();
    sp.dm_mass = mass;
    return OV_OK;
}

// Thick-restart Lanczos with full reorthogonalisation on A0 in sector chi at the phase (FP32 sign
// applications): Krylov bases of K vectors; after each pass the projected matrix (from the
// reorthogonalisation coefficients) gives Ritz pairs, and the lowest `keep` Ritz vectors plus the
// next Lanczos vector start the next pass, until the n_ev lowest Ritz estimates |beta y_K| are
// below tol or max_restarts passes ran.  Then Rayleigh-Ritz with A0 applied to the n_ev Ritz
// vectors; registers the space for (phase, chi).
int lanczos_overlap(ov_ctx* c, double phase, int chi, int n_ev, int K, double tol, int max_restarts,
                    cudaStream_t s) {
    const int V = c->g.V;
    const long long n12 = 12LL * V;
    const size_t vb = vec_bytes(c, OV_PREC_F32);
    const int keep = std::min(n_ev + std::max(8, n_ev / 2), K - 8);
    if (keep < n_ev) return fail(c, OV_ERR_ARG, "krylov = %d too small for n_ev = %d (needs >= n_ev + 8)", K, n_ev);
    void *Q, *w, *t, *r64, *Qr;
    TRY(workspace(c, "lz_Q", OV_PREC_F32, K + 1, &Q));
    TRY(workspace(c, "lz_Qr", OV_PREC_F32, keep, &Qr));
    TRY(workspace(c, "lz_w", OV_PREC_F32, 1, &w));
    TRY(workspace(c, "lz_t", OV_PREC_F32, 1, &t));
    TRY(workspace(c, "lz_r64", OV_PREC_F64, 1, &r64));
    SysSet S1;
    S1.n = 1;
    S1.phase = {phase};
    S1.chi = {(signed char)chi};
    TRY(ensure_small(c, (long long)(K + 1) * std::max(K, n_ev), (long long)(K + 1) * 4 * 152, std::max(n_ev, 1)));
    // start: a random vector of the sector, normalised
    random_fill_k<<<152 * 8, 256, 0, s>>>((double2*)r64, n12, 0x1a2c3e5dULL + (unsigned long long)(chi + 2), 0);
    count_launch();
    launch_convert<double, float>(r64, t, V, 1, s);
    const int zero = 0;
    CK(cudaMemcpyAsync(c->d_idx, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    const signed char ch = (signed char)chi;
    CK(cudaMemcpyAsync(c->d_chi, &ch, 1, cudaMemcpyHostToDevice, s));
    launch_chiral_split<float>(t, w, c->d_idx, c->d_chi, V, 1, s);
    CKL();
    double nrm2 = 0.0;
    norm2_rhs<float>(w, n12, 1, &nrm2, c->d_partial, c->d_red, s);
    launch_scale<float>(1.0 / std::sqrt(nrm2), w, Q, n12, s);
    std::vector<HostCplx> H((size_t)K * K, HostCplx{0, 0}), T, Y;  // H: projections, column-major
    std::vector<double> th, kept_theta;
    int kb = 0, passes = 0, steps = 0;
    double last_b = 0.0, worst_est = 0.0;
    // the operator only needs to be a tenth of the residual target accurate: the lowest degree
    // with delta <= tol / 10 (A0 W is recomputed in FP64 at the full degree afterwards)
    const int ldeg = degree_for_delta(c, 0.1 * tol);
    for (;;) {
        for (int j = kb; j < K; ++j) {
            char* qj = (char*)Q + (size_t)j * vb;
            TRY(sign_pipeline<float>(c, qj, S1, false, sector_operator(c, 0.0, qj), w, s, ldeg));
            ++steps;
            // w -= Q_{0..j} (Q^+ w), twice; the coefficients are column j of Q^+ A0 Q
            std::vector<HostCplx> gsum(j + 1, HostCplx{0, 0});
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<HostCplx> g;
                TRY(gram_host<float>(c, Q, j + 1, w, 1, g, s));
                TRY(dspace_combine(c, Q, j + 1, g, -1.0, w, t, s));
                std::swap(w, t);
                for (int i = 0; i <= j; ++i) {
                    gsum[i].re += g[i].re;
                    gsum[i].im += g[i].im;
                }
            }
            for (int i = 0; i <= j; ++i) H[i + (size_t)j * K] = gsum[i];
            double b2 = 0.0;
            norm2_rhs<float>(w, n12, 1, &b2, c->d_partial, c->d_red, s);
            last_b = std::sqrt(b2);
            if (!std::isfinite(last_b)) return fail(c, OV_ERR_NAN, "D_ov Lanczos: NaN at step %d", steps);
            if (!(last_b > 0.0)) return fail(c, OV_ERR_BREAKDOWN, "D_ov Lanczos: invariant subspace at step %d", steps);
            launch_scale<float>(1.0 / last_b, w, (char*)Q + (size_t)(j + 1) * vb, n12, s);
            CKL();
        }
        ++passes;
        // Hermitian projected matrix: kept Ritz values on the leading diagonal, the rest from the
        // columns computed in this pass
        T.assign((size_t)K * K, HostCplx{0, 0});
        for (int j = 0; j < K; ++j) {
            if (j < kb) T[j + (size_t)j * K] = HostCplx{kept_theta[j], 0.0};
            else T[j + (size_t)j * K] = HostCplx{H[j + (size_t)j * K].re, 0.0};
            for (int i = 0; i < j; ++i) {
                if (j < kb) continue;  // the kept block is diagonal
                const HostCplx h = H[i + (size_t)j * K];
                T[i + (size_t)j * K] = h;
                T[j + (size_t)i * K] = HostCplx{h.re, -h.im};
            }
        }
        host_eigh(K, T, th, Y);
        worst_est = 0.0;
        for (int i = 0; i < n_ev; ++i) {
            const HostCplx y = Y[(K - 1) + (size_t)i * K];
            worst_est = std::max(worst_est, last_b * std::sqrt(y.re * y.re + y.im * y.im));
        }
        if (worst_est <= tol || passes > max_restarts) break;
        // restart: Q[0..keep) = Q Y[:, 0..keep), Q[keep] = the next Lanczos vector
        std::vector<HostCplx> Yk(Y.begin(), Y.begin() + (size_t)K * keep);
        TRY(rotate<float>(c, Q, K, Yk, keep, Qr, s));
        CK(cudaMemcpyAsync(Q, Qr, vb * keep, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync((char*)Q + (size_t)keep * vb, (char*)Q + (size_t)K * vb, vb, cudaMemcpyDeviceToDevice, s));
        kept_theta.assign(th.begin(), th.begin() + keep);
        kb = keep;
        std::fill(H.begin(), H.end(), HostCplx{0, 0});
    }
    Y.resize((size_t)K * n_ev);  // the n_ev lowest Ritz vectors of the last pass
    DefSpace* sp = find_dspace(c, phase, chi);
    if (!sp) {
        c->dspaces.push_back(DefSpace());
        sp = &c->dspaces.back();
        sp->phase = phase;
        sp->chi = chi;
    }
    for (void** q : {&sp->W, &sp->AW0, &sp->AWm, &sp->W64, &sp->DW64, &sp->DmW64, &sp->AW64, &sp->AWm64})
        if (*q) {
            CK(cudaStreamSynchronize(s));
            CK(cudaFree(*q));
            *q = nullptr;
        }
    sp->n = 0;
    sp->mass = -1.0;
    sp->dm_mass = -1.0;
    if (cudaMalloc(&sp->W, vb * n_ev) != cudaSuccess || cudaMalloc(&sp->AW0, vb * n_ev) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "deflation space: allocation of %d vectors failed", n_ev);
    }
    TRY(rotate<float>(c, Q, K, Y, n_ev, sp->W, s));
    void* tmp;
    TRY(workspace(c, "lz_tmp", OV_PREC_F32, n_ev, &tmp));
    TRY(cholqr2<float>(c, sp->W, n_ev, tmp, s));
    // Rayleigh-Ritz with A0 on the Ritz vectors
    SysSet Sn;
    Sn.n = n_ev;
    Sn.phase.assign(n_ev, phase);
    Sn.chi.assign(n_ev, (signed char)chi);
    TRY(sign_pipeline<float>(c, sp->W, Sn, false, sector_operator(c, 0.0, sp->W), sp->AW0, s, ldeg));
    std::vector<HostCplx> Hr, Z;
    TRY(gram_host<float>(c, sp->W, n_ev, sp->AW0, n_ev, Hr, s));
    hermitize(Hr, n_ev);
    host_eigh(n_ev, Hr, sp->theta, Z);
    TRY(rotate<float>(c, sp->W, n_ev, Z, n_ev, tmp, s));
    CK(cudaMemcpyAsync(sp->W, tmp, vb * n_ev, cudaMemcpyDeviceToDevice, s));
    TRY(rotate<float>(c, sp->AW0, n_ev, Z, n_ev, tmp, s));
    CK(cudaMemcpyAsync(sp->AW0, tmp, vb * n_ev, cudaMemcpyDeviceToDevice, s));
    // residuals |A0 w_i - theta_i w_i|
    std::vector<double> mth(n_ev), ones(n_ev, 1.0);
    for (int i = 0; i < n_ev; ++i) mth[i] = -sp->theta[i];
    CK(cudaMemcpyAsync(tmp, sp->AW0, vb * n_ev, cudaMemcpyDeviceToDevice, s));
    launch_axpby<float>(mth.data(), sp->W, ones.data(), tmp, n12, n_ev, s);
    CKL();
    sp->res.assign(n_ev, 0.0);
    norm2_rhs<float>(tmp, n12, n_ev, sp->res.data(), c->d_partial, c->d_red, s);
    for (double& r : sp->res) r = std::sqrt(r);
    sp->n = n_ev;
    char buf[256];
    double worst = 0.0;
    for (double r : sp->res) worst = std::max(worst, r);
    snprintf(buf, sizeof(buf), "D_ov low modes: phase %.6g, chirality %+d, %d Lanczos steps (degree %d) in %d passes of %d, "
             "%d Ritz pairs in [%.3e, %.3e], worst residual %.2e (estimate %.2e)", phase, chi, steps, ldeg, passes, K,
             n_ev, sp->theta.front(), sp->theta.back(), worst, worst_est);
    c->info = buf;
    return OV_OK;
}

// W in FP64 and D_ov^+ W (FP64 sign applications, the full degree) for the solver's FP64 share.
int dspace_fp64(ov_ctx* c, DefSpace& sp, cudaStream_t s) {
    for (void** q : {&sp.W64, &sp.DW64, &sp.DmW64})
        if (*q) {
            CK(cudaStreamSynchronize(s));
            CK(cudaFree(*q));
            *q = nullptr;
        }
    sp.dm_mass = -1.0;
    const size_t b64 = vec_bytes(c, OV_PREC_F64) * sp.n;
    if (cudaMalloc(&sp.W64, b64) != cudaSuccess || cudaMalloc(&sp.DW64, b64) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "deflation space: allocation of %d FP64 vectors failed", sp.n);
    }
    launch_convert<float, double>(sp.W, sp.W64, c->g.V, sp.n, s);
    CKL();
    SysSet S;
    S.n = sp.n;
    S.phase.assign(sp.n, sp.phase);
    TRY(overlap_op<double>(c, sp.W64, S, 0.0, true, sp.DW64, s));
    // A0 W = 2 P_s D_ov^+ W in FP64; the FP32 copy replaces the FP32-operator one
    if (cudaMalloc(&sp.AW64, b64) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "deflation space: allocation of %d FP64 vectors failed", sp.n);
    }
    std::vector<int> idx(sp.n);
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<signed char> chis(sp.n, (signed char)sp.chi);
    TRY(ensure_small(c, 0, 0, sp.n));
    CK(cudaMemcpyAsync(c->d_idx, idx.data(), sizeof(int) * sp.n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->d_chi, chis.data(), sp.n, cudaMemcpyHostToDevice, s));
    void* t64;
    TRY(workspace(c, "dsp_t64", OV_PREC_F64, sp.n, &t64));
    launch_chiral_split<double>(sp.DW64, t64, c->d_idx, c->d_chi, c->g.V, sp.n, s);
    launch_scale<double>(2.0, t64, sp.AW64, 12LL * c->g.V * sp.n, s);
    launch_convert<double, float>(sp.AW64, sp.AW0, c->g.V, sp.n, s);
    CKL();
    sp.mass = -1.0;
    sp.Einv64.clear();
    // Ritz values and residuals of the full-degree operator: theta_i = w_i^+ A0 w_i,
    // |A0 w_i - theta_i w_i| (FP64)
    std::vector<HostCplx> H;
    TRY(gram_host<double>(c, sp.W64, sp.n, sp.AW64, sp.n, H, s));
    std::vector<double> mth(sp.n), ones(sp.n, 1.0);
    for (int i = 0; i < sp.n; ++i) {
        sp.theta[i] = H[i + (size_t)i * sp.n].re;
        mth[i] = -sp.theta[i];
    }
    CK(cudaMemcpyAsync(t64, sp.AW64, b64, cudaMemcpyDeviceToDevice, s));
    launch_axpby<double>(mth.data(), sp.W64, ones.data(), t64, 12LL * c->g.V, sp.n, s);
    CKL();
    norm2_rhs<double>(t64, 12LL * c->g.V, sp.n, sp.res.data(), c->d_partial, c->d_red, s);
    for (double& r : sp.res) r = std::sqrt(r);
    return OV_OK;
}

// CG on the chiral-sector normal operator A_s = P_s [2 (1 - m^2/4)(1 + s sign) + m^2] P_s for each
// system (rhs vector B_k in sector chi_k), in precision R (ST: storage of the polynomial loop's
// links and vectors, R or a 16-bit format with R = float).  Y: solutions, in the order of S.
// Converged systems leave the batch: the active ones are kept at the front (a converged
// system is swapped with the last active one), so later sign applications run only on
// systems that still iterate; Y is put back in the original order at the end.
// coef0 (optional, FP32): for each system whose space carries the FP64 part, the Galerkin start is
// returned as coefficients c (y = W c + Y) instead of being added to Y in FP32: its size, about
// |r| / lambda_min, would leave FP32 rounding of that order in Y.
template <typename R, typename ST = R>
int inner_cg(ov_ctx* c, double mass, const SysSet& S0, const void* B, void* Y, const std::vector<double>& tol_rel0,
             int max_iter, int* iters, cudaStream_t s, int degree = 0,
             std::vector<std::vector<HostCplx>>* coef0 = nullptr) {
    constexpr bool F64 = std::is_same<R, double>::value;
    const int prec = prec_of<R>();
    const int ns = S0.n;
    const long long n12 = 12LL * c->g.V;
    void *r, *p, *Ap, *tmp;
    TRY(workspace(c, "cg_r", prec, ns, &r));
    TRY(workspace(c, "cg_p", prec, ns, &p));
    TRY(workspace(c, "cg_Ap", prec, ns, &Ap));
    TRY(workspace(c, "cg_tmp", prec, ns, &tmp));
    const size_t vb = vec_bytes(c, prec);
    const size_t bytes = vb * ns;
    CK(cudaMemcpyAsync(r, B, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p, B, bytes, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(Y, 0, bytes, s));
    TRY(ensure_small(c, 0, (long long)kRedBlocks * ns, ns));
    SysSet S = S0;
    std::vector<double> tol_rel = tol_rel0;
    std::vector<int> perm(ns);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<double> rr(ns), rr_new(ns), b2(ns), alpha(ns), beta(ns), ones(ns, 1.0);
    std::vector<double2> pap(ns);
    // 16-bit storage: the operator carries rounding of ~1e-3 that differs between applications, so
    // the CG residual stalls near that level; a system whose best residual has not halved within
    // kStall iterations leaves the batch (the outer FP64 loop continues from its iterate)
    constexpr bool HALF = !std::is_same<R, ST>::value;
    constexpr int kStall = 100;
    std::vector<double> best(ns, 0.0);
    std::vector<int> best_it(ns, 0);
    int stalled = 0;
    norm2_rhs<R>(r, n12, ns, rr.data(), c->d_partial, c->d_red, s);
    b2 = rr;
    // Deflation with the D_ov low modes of each system's (phase, chirality), in the CG's precision
    // (FP32 vectors, or their FP64 counterparts W, A(m) W for an FP64 CG): start from the Galerkin
    // solution on the space, y = W E^-1 W^+ b (E = W^+ A W), and keep the search directions
    // A-orthogonal to it, p = r + beta p - W E^-1 (A W)^+ r (deflated CG).
    std::vector<DefSpace*> dsp(ns, nullptr);
    bool any_defl = false;
    auto Wof = [](DefSpace* sp) -> const void* { return F64 ? sp->W64 : sp->W; };
    auto AWof = [](DefSpace* sp) -> const void* { return F64 ? sp->AWm64 : sp->AWm; };
    for (int k = 0; k < ns; ++k) {
        DefSpace* sp = S0.chi.empty() ? nullptr : find_dspace(c, S0.phase[k], S0.chi[k]);
        if (!sp || !(rr[k] > 0.0)) continue;
        if (F64) {
            if (!sp->AW64) continue;  // no FP64 data for this space
            TRY(dspace_prepare64(c, *sp, mass, s));
        } else {
            TRY(dspace_prepare(c, *sp, mass, s));
        }
        char* bk = (char*)B + (size_t)k * vb;
        char* rk = (char*)r + (size_t)k * vb;
        std::vector<HostCplx> dco, mu;
        TRY(dspace_coeffs<R>(c, *sp, Wof(sp), bk, dco, true, s));
        if (!F64 && coef0 && sp->DW64) (*coef0)[k] = dco;  // kept in FP64 by the caller
        else TRY(dspace_combine<R>(c, Wof(sp), sp->n, dco, 1.0, nullptr, (char*)Y + (size_t)k * vb, s));
        TRY(dspace_combine<R>(c, AWof(sp), sp->n, dco, -1.0, bk, rk, s));
        TRY(dspace_coeffs<R>(c, *sp, AWof(sp), rk, mu, true, s));
        TRY(dspace_combine<R>(c, Wof(sp), sp->n, mu, -1.0, rk, (char*)p + (size_t)k * vb, s));
        dsp[k] = sp;
        any_defl = true;
    }
    if (any_defl) norm2_rhs<R>(r, n12, ns, rr.data(), c->d_partial, c->d_red, s);
    auto swap_vec = [&](void* base, int i, int j) -> int {
        char* bi = (char*)base + (size_t)i * vb;
        char* bj = (char*)base + (size_t)j * vb;
        CK(cudaMemcpyAsync(tmp, bi, vb, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bi, bj, vb, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bj, tmp, vb, cudaMemcpyDeviceToDevice, s));
        return OV_OK;
    };
    // drop position k from the active front [0, na)
    auto retire = [&](int k, int& na) -> int {
        const int last = na - 1;
        if (k != last) {
            TRY(swap_vec(r, k, last));
            TRY(swap_vec(p, k, last));
            TRY(swap_vec(Y, k, last));
            std::swap(perm[k], perm[last]);
            std::swap(rr[k], rr[last]);
            std::swap(b2[k], b2[last]);
            std::swap(tol_rel[k], tol_rel[last]);
            std::swap(S.phase[k], S.phase[last]);
            std::swap(S.chi[k], S.chi[last]);
            std::swap(dsp[k], dsp[last]);
            std::swap(best[k], best[last]);
            std::swap(best_it[k], best_it[last]);
        }
        --na;
        return OV_OK;
    };
    int na = ns;
    for (int k = na - 1; k >= 0; --k)
        if (!(rr[k] > 0.0)) TRY(retire(k, na));
    const double k1 = 2.0 * (1.0 - 0.25 * mass * mass);
    Epilogue fin;
    fin.c_op = k1 / c->hw_norm;
    fin.c1 = k1;
    fin.chi = c->d_chi;
    fin.c2 = k1 + mass * mass;
    fin.v2 = p;
    int it = 0;
    for (it = 0; it < max_iter && na > 0; ++it) {
        SysSet A;
        A.n = na;
        A.phase.assign(S.phase.begin(), S.phase.begin() + na);
        A.chi.assign(S.chi.begin(), S.chi.begin() + na);
        TRY((sign_pipeline<R, ST>(c, p, A, false, fin, Ap, s, degree)));
        dot_rhs<R>(p, Ap, n12, na, pap.data(), c->d_partial, c->d_red, s);
        for (int k = 0; k < na; ++k) {
            if (!std::isfinite(pap[k].x) || !std::isfinite(rr[k]))
                return fail(c, OV_ERR_NAN, "inner CG: NaN/Inf in <p, A p> (system %d, iteration %d)", perm[k], it);
            if (pap[k].x <= 0.0)
                return fail(c, OV_ERR_BREAKDOWN, "inner CG: <p, A p> = %g <= 0 (system %d, iteration %d)", pap[k].x,
                            perm[k], it);
            alpha[k] = rr[k] / pap[k].x;
        }
        launch_cg_xr<R>(alpha.data(), p, Ap, Y, r, n12, na, s);
        CKL();
        norm2_rhs<R>(r, n12, na, rr_new.data(), c->d_partial, c->d_red, s);
        for (int k = 0; k < na; ++k) {
            beta[k] = rr_new[k] / rr[k];
            rr[k] = rr_new[k];
        }
        if (!any_defl) {
            launch_axpby<R>(ones.data(), r, beta.data(), p, n12, na, s);  // p = r + beta p
        } else {
            for (int k = 0; k < na; ++k) {
                char* rk = (char*)r + (size_t)k * vb;
                char* pk = (char*)p + (size_t)k * vb;
                const void* dir = rk;
                if (dsp[k]) {  // r - W E^-1 (A W)^+ r
                    std::vector<HostCplx> mu;
                    TRY(dspace_coeffs<R>(c, *dsp[k], AWof(dsp[k]), rk, mu, true, s));
                    char* tk = (char*)tmp + (size_t)k * vb;
                    TRY(dspace_combine<R>(c, Wof(dsp[k]), dsp[k]->n, mu, -1.0, rk, tk, s));
                    dir = tk;
                }
                launch_axpby<R>(&ones[k], dir, &beta[k], pk, n12, 1, s);
            }
        }
        CKL();
        for (int k = na - 1; k >= 0; --k) {
            if (std::sqrt(rr[k]) <= tol_rel[k] * std::sqrt(b2[k])) {
                TRY(retire(k, na));
                continue;
            }
            if (HALF) {
                if (best[k] == 0.0 || rr[k] < 0.25 * best[k]) {  // |r| halved: a new reference point
                    best[k] = rr[k];
                    best_it[k] = it;
                } else if (it - best_it[k] >= kStall) {
                    ++stalled;
                    TRY(retire(k, na));
                }
            }
        }
    }
    *iters = it;
    if (stalled) c->cg_stalls += stalled;
    // back to the original order: position k holds system perm[k]
    bool moved = false;
    for (int k = 0; k < ns; ++k) moved = moved || perm[k] != k;
    if (moved) {
        void* Yo;
        TRY(workspace(c, "cg_yorder", prec, ns, &Yo));
        for (int k = 0; k < ns; ++k)
            CK(cudaMemcpyAsync((char*)Yo + (size_t)perm[k] * vb, (char*)Y + (size_t)k * vb, vb,
                               cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(Y, Yo, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return na > 0 ? OV_ERR_NOT_CONVERGED : OV_OK;
}

// Multi-shift CG: the multi-mass CG of Sec. 3.2.  The chiral-sector operators of all masses form
// one shifted family, A(m) = k(m) (A0 + sigma(m)) with A0 = P_s 2 (1 + s sign) P_s, k(m) = 1 - m^2/4
// and sigma(m) = m^2 / k(m).  With M = A(m_b) of the lightest mass,
// A(m_i) = (k_i / k_b) (M + tau_i), tau_i = k_b (sigma_i - sigma_b) >= 0, so one Krylov space of M
// serves every mass: each shifted residual stays parallel to the seed's, r_i = zeta_i r, and
// zeta_i, alpha_i and beta_i follow from the seed's alpha and beta by scalar recurrences
// (Jegerlehner, hep-lat/9612014).  One sign application per iteration and system, whatever the
// number of masses.  Z is [mass][system]; Z[i][k] returns A(m_i)^{-1} B_k (the factor k_b / k_i
// applied).  A shift whose residual |zeta_i| |r| meets its system's tolerance stops updating; a
// system leaves the batch when its seed (the lightest mass, the last to converge) does.
template <typename R, typename ST = R>
int inner_cg_shifted(ov_ctx* c, const std::vector<double>& mass, const SysSet& S0, const void* B, void* Z,
                     const std::vector<double>& tol_rel0, int max_iter, int* iters, cudaStream_t s, int degree) {
    const int prec = prec_of<R>();
    const int ns = S0.n, nm = (int)mass.size();
    const long long n12 = 12LL * c->g.V;
    const size_t vb = vec_bytes(c, prec);
    const size_t bytes = vb * ns;
    int ib = 0;
    for (int i = 1; i < nm; ++i)
        if (std::fabs(mass[i]) < std::fabs(mass[ib])) ib = i;
    const double mb2 = mass[ib] * mass[ib];
    const double kb = 1.0 - 0.25 * mb2;
    std::vector<double> tau(nm);
    for (int i = 0; i < nm; ++i) {
        const double m2 = mass[i] * mass[i];
        tau[i] = kb * (m2 / (1.0 - 0.25 * m2) - mb2 / kb);
    }
    void *r, *Ap, *tmp, *P;
    TRY(workspace(c, "mcg_r", prec, ns, &r));
    TRY(workspace(c, "mcg_Ap", prec, ns, &Ap));
    TRY(workspace(c, "mcg_tmp", prec, 1, &tmp));
    TRY(workspace(c, "mcg_p", prec, (long long)nm * ns, &P));
    auto at = [&](void* base, int i, int k) { return (char*)base + ((size_t)i * ns + k) * vb; };
    CK(cudaMemcpyAsync(r, B, bytes, cudaMemcpyDeviceToDevice, s));
    for (int i = 0; i < nm; ++i) {
        CK(cudaMemcpyAsync(at(P, i, 0), B, bytes, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(at(Z, i, 0), 0, bytes, s));
    }
    TRY(ensure_small(c, 0, (long long)kRedBlocks * ns, ns));
    SysSet S = S0;
    std::vector<double> tol_rel = tol_rel0;
    std::vector<int> perm(ns);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<double> rr(ns), rr_new(ns), b2(ns), alpha(ns), beta(ns), ones(ns, 1.0);
    std::vector<double> a_prev(ns, 1.0), b_prev(ns, 0.0), ca(ns), cb(ns);
    // per (mass, system), index i * ns + k: zeta_k, zeta_{k-1}, zeta_{k+1}; frozen once converged
    std::vector<double> z((size_t)nm * ns, 1.0), zp((size_t)nm * ns, 1.0), zn((size_t)nm * ns, 1.0);
    std::vector<char> frozen((size_t)nm * ns, 0);
    std::vector<double2> pap(ns);
    norm2_rhs<R>(r, n12, ns, rr.data(), c->d_partial, c->d_red, s);
    b2 = rr;
    auto swap_vec = [&](char* bi, char* bj) -> int {
        CK(cudaMemcpyAsync(tmp, bi, vb, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bi, bj, vb, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(bj, tmp, vb, cudaMemcpyDeviceToDevice, s));
        return OV_OK;
    };
    // drop position k from the active front [0, na)
    auto retire = [&](int k, int& na) -> int {
        const int last = na - 1;
        if (k != last) {
            TRY(swap_vec((char*)r + (size_t)k * vb, (char*)r + (size_t)last * vb));
            for (int i = 0; i < nm; ++i) {
                TRY(swap_vec(at(P, i, k), at(P, i, last)));
                TRY(swap_vec(at(Z, i, k), at(Z, i, last)));
                const size_t q = (size_t)i * ns + k, ql = (size_t)i * ns + last;
                std::swap(z[q], z[ql]);
                std::swap(zp[q], zp[ql]);
                std::swap(frozen[q], frozen[ql]);
            }
            std::swap(perm[k], perm[last]);
            std::swap(rr[k], rr[last]);
            std::swap(b2[k], b2[last]);
            std::swap(tol_rel[k], tol_rel[last]);
            std::swap(a_prev[k], a_prev[last]);
            std::swap(b_prev[k], b_prev[last]);
            std::swap(S.phase[k], S.phase[last]);
            std::swap(S.chi[k], S.chi[last]);
        }
        --na;
        return OV_OK;
    };
    int na = ns;
    for (int k = na - 1; k >= 0; --k)
        if (!(rr[k] > 0.0)) TRY(retire(k, na));
    const double k1 = 2.0 * kb;
    Epilogue fin;
    fin.c_op = k1 / c->hw_norm;
    fin.c1 = k1;
    fin.chi = c->d_chi;
    fin.c2 = k1 + mb2;
    int it = 0;
    for (it = 0; it < max_iter && na > 0; ++it) {
        SysSet A;
        A.n = na;
        A.phase.assign(S.phase.begin(), S.phase.begin() + na);
        A.chi.assign(S.chi.begin(), S.chi.begin() + na);
        void* pb = at(P, ib, 0);
        fin.v2 = pb;
        TRY((sign_pipeline<R, ST>(c, pb, A, false, fin, Ap, s, degree)));  // Ap = M p (seed direction)
        dot_rhs<R>(pb, Ap, n12, na, pap.data(), c->d_partial, c->d_red, s);
        for (int k = 0; k < na; ++k) {
            if (!std::isfinite(pap[k].x) || !std::isfinite(rr[k]))
                return fail(c, OV_ERR_NAN, "multi-mass CG: NaN/Inf in <p, M p> (system %d, iteration %d)", perm[k], it);
            if (pap[k].x <= 0.0)
                return fail(c, OV_ERR_BREAKDOWN, "multi-mass CG: <p, M p> = %g <= 0 (system %d, iteration %d)",
                            pap[k].x, perm[k], it);
            alpha[k] = rr[k] / pap[k].x;
        }
        // zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} / (a_k b_{k-1} (zeta_{k-1} - zeta_k) + zeta_{k-1} a_{k-1} (1 + tau a_k));
        // x_i += (a_k zeta_{k+1} / zeta_k) p_i
        for (int i = 0; i < nm; ++i) {
            for (int k = 0; k < na; ++k) {
                const size_t q = (size_t)i * ns + k;
                ca[k] = 0.0;
                if (frozen[q]) continue;
                const double den = alpha[k] * b_prev[k] * (zp[q] - z[q]) + zp[q] * a_prev[k] * (1.0 + tau[i] * alpha[k]);
                zn[q] = z[q] * zp[q] * a_prev[k] / den;
                if (!std::isfinite(zn[q]) || zn[q] == 0.0)
                    return fail(c, OV_ERR_BREAKDOWN, "multi-mass CG: shift recurrence broke down (mass %d, system %d)",
                                i, perm[k]);
                ca[k] = alpha[k] * zn[q] / z[q];
            }
            launch_axpby<R>(ca.data(), at(P, i, 0), ones.data(), at(Z, i, 0), n12, na, s);
        }
        for (int k = 0; k < na; ++k) ca[k] = -alpha[k];
        launch_axpby<R>(ca.data(), Ap, ones.data(), r, n12, na, s);  // r -= alpha M p
        CKL();
        norm2_rhs<R>(r, n12, na, rr_new.data(), c->d_partial, c->d_red, s);
        for (int k = 0; k < na; ++k) beta[k] = rr_new[k] / rr[k];
        // p_i = zeta_{k+1} r + beta (zeta_{k+1} / zeta_k)^2 p_i
        for (int i = 0; i < nm; ++i) {
            for (int k = 0; k < na; ++k) {
                const size_t q = (size_t)i * ns + k;
                if (frozen[q]) {
                    ca[k] = 0.0;
                    cb[k] = 1.0;
                    continue;
                }
                const double t = zn[q] / z[q];
                ca[k] = zn[q];
                cb[k] = beta[k] * t * t;
            }
            launch_axpby<R>(ca.data(), r, cb.data(), at(P, i, 0), n12, na, s);
        }
        CKL();
        for (int k = 0; k < na; ++k) {
            for (int i = 0; i < nm; ++i) {
                const size_t q = (size_t)i * ns + k;
                if (frozen[q]) continue;
                zp[q] = z[q];
                z[q] = zn[q];
            }
            a_prev[k] = alpha[k];
            b_prev[k] = beta[k];
            rr[k] = rr_new[k];
            for (int i = 0; i < nm; ++i) {
                const size_t q = (size_t)i * ns + k;
                if (!frozen[q] && std::fabs(z[q]) * std::sqrt(rr[k]) <= tol_rel[k] * std::sqrt(b2[k])) frozen[q] = 1;
            }
        }
        for (int k = na - 1; k >= 0; --k)
            if (frozen[(size_t)ib * ns + k]) TRY(retire(k, na));
    }
    *iters = it;
    // back to the original order (position k holds system perm[k]) and A(m_i)^-1 = (k_b / k_i) (M + tau_i)^-1
    bool moved = false;
    for (int k = 0; k < ns; ++k) moved = moved || perm[k] != k;
    void* Zo = nullptr;
    if (moved) TRY(workspace(c, "mcg_zorder", prec, ns, &Zo));
    for (int i = 0; i < nm; ++i) {
        if (moved) {
            for (int k = 0; k < ns; ++k)
                CK(cudaMemcpyAsync((char*)Zo + (size_t)perm[k] * vb, at(Z, i, k), vb, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(at(Z, i, 0), Zo, bytes, cudaMemcpyDeviceToDevice, s));
        }
        launch_scale<R>(kb / (1.0 - 0.25 * mass[i] * mass[i]), at(Z, i, 0), at(Z, i, 0), n12 * ns, s);
    }
    CKL();
    return na > 0 ? OV_ERR_NOT_CONVERGED : OV_OK;
}

// Relative tolerance of an inner solve when the caller set none: FP64 the outer target itself, FP32
// 1e-6, and above the operator's own rounding for the 16-bit formats (FP16 1e-2, BF16 3e-2: one sign
// application carries ~2e-3 / ~1e-2 relative error at these degrees).
template <typename R, typename ST>
double inner_base_tol(const ov_ctx* c) {
    if (c->p.inner_tol > 0.0) return c->p.inner_tol;
    if (std::is_same<R, double>::value) return 0.0;
    if (std::is_same<ST, H16>::value) return 1e-2;
    if (std::is_same<ST, B16>::value) return 3e-2;
    return 1e-6;
}

// R: arithmetic of the inner CG and its correction (FP64 or FP32); ST: storage of their polynomial
// loops (R, or FP16 / BF16 with R = float).  The true residual and x stay FP64.
template <typename R, typename ST = R>
int solve_impl(ov_ctx* c, double mass, const SysSet& Srhs, const void* b, void* x, double tol, ov_solve_stats* st,
               cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    const int nrhs = Srhs.n;
    const int V = c->g.V;
    const long long n12 = 12LL * V;
    const int prec = prec_of<R>();
    const size_t vb64 = vec_bytes(c, OV_PREC_F64);
    void *B, *X, *Rr, *DX, *S64, *Bs, *Ys, *Ysum, *E, *E64;
    TRY(workspace(c, "sol_B", OV_PREC_F64, nrhs, &B));
    TRY(workspace(c, "sol_X", OV_PREC_F64, nrhs, &X));
    TRY(workspace(c, "sol_R", OV_PREC_F64, nrhs, &Rr));
    TRY(workspace(c, "sol_DX", OV_PREC_F64, nrhs, &DX));
    TRY(workspace(c, "sol_S64", OV_PREC_F64, 2 * nrhs, &S64));
    TRY(workspace(c, "sol_Bs", prec, 2 * nrhs, &Bs));
    TRY(workspace(c, "sol_Ys", prec, 2 * nrhs, &Ys));
    TRY(workspace(c, "sol_Ysum", prec, nrhs, &Ysum));
    TRY(workspace(c, "sol_E", prec, nrhs, &E));
    TRY(workspace(c, "sol_E64", OV_PREC_F64, nrhs, &E64));
    TRY(ensure_small(c, 0, (long long)kRedBlocks * 2 * nrhs, 2 * nrhs));
    launch_pack_spinor<double>(b, OV_C128, B, V, nrhs, s);
    launch_pack_spinor<double>(x, OV_C128, X, V, nrhs, s);
    CKL();
    const long long dslash0 = c->dslash_count, sign0 = c->sign_count;
    std::vector<double> bn2(nrhs), xn2(nrhs), rn2(nrhs), res(nrhs, 0.0);
    norm2_rhs<double>(B, n12, nrhs, bn2.data(), c->d_partial, c->d_red, s);
    norm2_rhs<double>(X, n12, nrhs, xn2.data(), c->d_partial, c->d_red, s);
    for (int j = 0; j < nrhs; ++j)
        if (!std::isfinite(bn2[j]) || !std::isfinite(xn2[j])) return fail(c, OV_ERR_NAN, "NaN/Inf in b or x (rhs %d)", j);
    std::vector<double> ones(nrhs, 1.0), mones(nrhs, -1.0);
    auto true_residual = [&]() -> int {
        TRY(overlap_op<double>(c, X, Srhs, mass, false, DX, s));
        CK(cudaMemcpyAsync(Rr, B, vb64 * nrhs, cudaMemcpyDeviceToDevice, s));
        launch_axpby<double>(mones.data(), DX, ones.data(), Rr, n12, nrhs, s);  // R = B - D X
        CKL();
        norm2_rhs<double>(Rr, n12, nrhs, rn2.data(), c->d_partial, c->d_red, s);
        for (int j = 0; j < nrhs; ++j) {
            if (!std::isfinite(rn2[j])) return fail(c, OV_ERR_NAN, "NaN/Inf in the true residual (rhs %d)", j);
            res[j] = bn2[j] > 0.0 ? std::sqrt(rn2[j] / bn2[j]) : 0.0;
        }
        return OV_OK;
    };
    bool xzero = true;
    for (int j = 0; j < nrhs; ++j) xzero = xzero && xn2[j] == 0.0;
    if (xzero) {
        CK(cudaMemcpyAsync(Rr, B, vb64 * nrhs, cudaMemcpyDeviceToDevice, s));
        for (int j = 0; j < nrhs; ++j) res[j] = bn2[j] > 0.0 ? 1.0 : 0.0;
        rn2 = bn2;
    } else {
        TRY(true_residual());
    }
    const double base_tol = inner_base_tol<R, ST>(c);
    int outer = 0, inner_total = 0, status = OV_OK;
    std::string hist = "solve:";
    const int max_outer = 60;
    while (true) {
        double worst = 0.0;
        for (int j = 0; j < nrhs; ++j) worst = std::max(worst, res[j]);
        if (worst <= tol) break;
        if (outer >= max_outer || inner_total >= c->p.max_iter) {
            status = OV_ERR_NOT_CONVERGED;
            break;
        }
        // chiral sectors of the residuals of the unconverged right-hand sides
        std::vector<int> src, sys_of_rhs(2 * nrhs, -1);
        std::vector<signed char> chi;
        for (int j = 0; j < nrhs; ++j)
            if (res[j] > tol)
                for (int sg = 0; sg < 2; ++sg) {
                    src.push_back(j);
                    chi.push_back(sg == 0 ? 1 : -1);
                }
        const int ns0 = (int)src.size();
        CK(cudaMemcpyAsync(c->d_idx, src.data(), sizeof(int) * ns0, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->d_chi, chi.data(), ns0, cudaMemcpyHostToDevice, s));
        launch_chiral_split<double>(Rr, S64, c->d_idx, c->d_chi, V, ns0, s);
        CKL();
        std::vector<double> sn2(ns0);
        norm2_rhs<double>(S64, n12, ns0, sn2.data(), c->d_partial, c->d_red, s);
        // keep the non-zero sectors, compacted
        SysSet S;
        std::vector<double> tol_rel;
        std::vector<int> rhs_of_sys;
        int ns = 0;
        for (int k = 0; k < ns0; ++k) {
            const int j = src[k];
            // a sector whose residual is below a quarter of the target cannot matter
            if (!(sn2[k] > 0.0) || std::sqrt(sn2[k]) <= 0.25 * tol * std::sqrt(bn2[j])) continue;
            if (ns != k)
                CK(cudaMemcpyAsync((char*)S64 + (size_t)ns * vb64, (char*)S64 + (size_t)k * vb64, vb64,
                                   cudaMemcpyDeviceToDevice, s));
            S.phase.push_back(Srhs.phase[j]);
            S.chi.push_back(chi[k]);
            sys_of_rhs[2 * j + (chi[k] > 0 ? 0 : 1)] = ns;
            rhs_of_sys.push_back(j);
            const double want = 0.5 * tol * std::sqrt(bn2[j] / sn2[k]);
            tol_rel.push_back(std::min(0.5, std::max(base_tol, want)));
            ++ns;
        }
        S.n = ns;
        // FP32 inner solves: each sector residual loses its part on the system's D_ov deflation
        // space in FP64, r_s -= A W c with c = (W^+ A W)^{-1} W^+ r_s (A, W in FP64); the FP32
        // CG then solves for the remainder, and W c enters the correction in FP64.
        std::vector<std::vector<HostCplx>> c_low(ns);
        if (std::is_same<R, float>::value) {
            for (int k = 0; k < ns; ++k) {
                DefSpace* sp = find_dspace(c, S.phase[k], S.chi[k]);
                if (!sp || !sp->AW64) continue;
                TRY(dspace_prepare64(c, *sp, mass, s));
                char* rk = (char*)S64 + (size_t)k * vb64;
                std::vector<HostCplx> g;
                TRY(gram_host<double>(c, sp->W64, sp->n, rk, 1, g, s));
                const int n = sp->n;
                c_low[k].assign(n, HostCplx{0, 0});
                for (int i = 0; i < n; ++i)
                    for (int q = 0; q < n; ++q) {
                        const HostCplx e = sp->Einv64[i + (size_t)q * n], x = g[q];
                        c_low[k][i].re += e.re * x.re - e.im * x.im;
                        c_low[k][i].im += e.re * x.im + e.im * x.re;
                    }
                void* t64;
                TRY(workspace(c, "sol_t64", OV_PREC_F64, 1, &t64));
                TRY(dspace_combine<double>(c, sp->AWm64, n, c_low[k], -1.0, rk, t64, s));
                CK(cudaMemcpyAsync(rk, t64, vb64, cudaMemcpyDeviceToDevice, s));
                double h2 = 0.0;
                norm2_rhs<double>(rk, n12, 1, &h2, c->d_partial, c->d_red, s);
                const int j = rhs_of_sys[k];
                if (h2 > 0.0) tol_rel[k] = std::min(0.5, std::max(base_tol, 0.5 * tol * std::sqrt(bn2[j] / h2)));
            }
        }
        if (std::is_same<R, double>::value)
            CK(cudaMemcpyAsync(Bs, S64, vb64 * ns, cudaMemcpyDeviceToDevice, s));
        else
            launch_convert<double, float>(S64, Bs, V, ns, s);
        CKL();
        // Degree of this cycle's polynomial (adaptive order, Sec. 3.2): a polynomial error delta
        // in the correction changes the corrected residual by about delta / m of the current one
        // (|D(m)^-1| ~ 1/m), so a cycle whose smallest inner tolerance is g needs delta <= eta m g,
        // eta = 0.5; the true residual keeps the full degree.
        int degree = 0;
        if (c->p.adaptive_order && ns > 0) {
            double g = 1.0;
            for (double t : tol_rel) g = std::min(g, t);
            degree = degree_for_delta(c, 0.5 * std::fabs(mass) * g);
        }
        int iters = 0;
        const long long stalls0 = c->cg_stalls;
        std::vector<std::vector<HostCplx>> coef0(ns);
        int rc = inner_cg<R, ST>(c, mass, S, Bs, Ys, tol_rel, c->p.max_iter - inner_total, &iters, s, degree, &coef0);
        for (int k = 0; k < ns; ++k) {
            if (c_low[k].empty()) continue;
            if (coef0[k].empty()) coef0[k].assign(c_low[k].size(), HostCplx{0, 0});
            for (size_t i = 0; i < c_low[k].size(); ++i) {
                coef0[k][i].re += c_low[k][i].re;
                coef0[k][i].im += c_low[k][i].im;
            }
        }
        inner_total += iters;
        if (rc != OV_OK && rc != OV_ERR_NOT_CONVERGED) {
            status = rc;
            break;
        }
        // y_j = y_{j,+} + y_{j,-};  e_j = D(m)^+ y_j;  x_j += e_j
        CK(cudaMemcpyAsync(c->d_idx, sys_of_rhs.data(), sizeof(int) * 2 * nrhs, cudaMemcpyHostToDevice, s));
        {
            dim3 grid(std::min<long long>((n12 + 255) / 256, 152 * 4), nrhs);
            merge_sectors_k<R><<<grid, 256, 0, s>>>((const typename C2<R>::T*)Ys, c->d_idx,
                                                    (typename C2<R>::T*)Ysum, n12);
            count_launch();
            CKL();
        }
        TRY((overlap_op<R, ST>(c, Ysum, Srhs, mass, true, E, s, degree)));
        if (std::is_same<R, double>::value)
            CK(cudaMemcpyAsync(E64, E, vb64 * nrhs, cudaMemcpyDeviceToDevice, s));
        else
            launch_convert<float, double>(E, E64, V, nrhs, s);
        // the deflation spaces' share of the correction, D(m)^+ W c, in FP64
        for (int k = 0; k < ns; ++k) {
            if (coef0[k].empty()) continue;
            DefSpace* sp = find_dspace(c, S.phase[k], S.chi[k]);
            TRY(dspace_prepare_dm(c, *sp, mass, s));
            void* t64;
            TRY(workspace(c, "sol_t64", OV_PREC_F64, 1, &t64));
            char* ej = (char*)E64 + (size_t)rhs_of_sys[k] * vb64;
            TRY(dspace_combine<double>(c, sp->DmW64, sp->n, coef0[k], 1.0, ej, t64, s));
            CK(cudaMemcpyAsync(ej, t64, vb64, cudaMemcpyDeviceToDevice, s));
        }
        launch_axpby<double>(ones.data(), E64, ones.data(), X, n12, nrhs, s);
        CKL();
        ++outer;
        // The new residual b - D(m) (x + e) = r - D(m) e.  While r is large, D(m) (x + e) is applied in
        // FP64.  Once every |r_j| <= theta |b_j| (FP32 and 16-bit inner precisions), the FP64 sum
        // r - D(m) e takes D(m) e from two FP32 applications, to e_hi = fl32(e) and e_lo = fl32(e - e_hi)
        // (so e itself enters to 2^-48): their rounding is about 1e-6 of |D(m) e| ~ |r|, below tol / 10
        // for theta = min(1e-5, 1e5 tol), and two FP32 applications cost a fifth of one FP64 application
        // on this GPU.
        double worst_prev = 0.0;
        for (int j = 0; j < nrhs; ++j) worst_prev = std::max(worst_prev, res[j]);
        const double theta = std::min(1e-5, 1e5 * tol);
        const bool fp32_update = std::is_same<R, float>::value && worst_prev <= theta;  // FP64 solves stay FP64
        if (fp32_update) {
            void *e32, *de32, *t64;
            TRY(workspace(c, "sol_e32", OV_PREC_F32, 2 * nrhs, &e32));
            TRY(workspace(c, "sol_de32", OV_PREC_F32, 2 * nrhs, &de32));
            TRY(workspace(c, "sol_t64", OV_PREC_F64, nrhs, &t64));
            const size_t vb32 = vec_bytes(c, OV_PREC_F32);
            char* e_lo = (char*)e32 + vb32 * nrhs;
            launch_convert<double, float>(E64, e32, V, nrhs, s);   // e_hi
            launch_convert<float, double>(e32, t64, V, nrhs, s);
            launch_axpby<double>(ones.data(), E64, mones.data(), t64, n12, nrhs, s);  // e - e_hi
            launch_convert<double, float>(t64, e_lo, V, nrhs, s);  // e_lo
            CKL();
            SysSet S2 = Srhs;
            S2.n = 2 * nrhs;
            S2.phase.insert(S2.phase.end(), Srhs.phase.begin(), Srhs.phase.end());
            TRY(overlap_op<float>(c, e32, S2, mass, false, de32, s));
            launch_convert<float, double>(de32, DX, V, nrhs, s);
            launch_axpby<double>(mones.data(), DX, ones.data(), Rr, n12, nrhs, s);  // R -= D e_hi
            launch_convert<float, double>((char*)de32 + vb32 * nrhs, DX, V, nrhs, s);
            launch_axpby<double>(mones.data(), DX, ones.data(), Rr, n12, nrhs, s);  // R -= D e_lo
            CKL();
            norm2_rhs<double>(Rr, n12, nrhs, rn2.data(), c->d_partial, c->d_red, s);
            for (int j = 0; j < nrhs; ++j) {
                if (!std::isfinite(rn2[j])) return fail(c, OV_ERR_NAN, "NaN/Inf in the updated residual (rhs %d)", j);
                res[j] = bn2[j] > 0.0 ? std::sqrt(rn2[j] / bn2[j]) : 0.0;
            }
        } else {
            TRY(true_residual());
        }
        {
            double worst = 0.0;
            for (int j = 0; j < nrhs; ++j) worst = std::max(worst, res[j]);
            char buf[128];
            snprintf(buf, sizeof(buf), " | cycle %d: n %d, %d inner, %d systems%s, residual %.2e%s", outer,
                     degree > 0 ? degree : c->p.poly_degree, iters, ns,
                     c->cg_stalls > stalls0 ? " (stalled)" : "", worst, fp32_update ? " (r - D e, D e in FP32)" : "");
            hist += buf;
        }
    }
    launch_unpack_spinor<double>(X, x, OV_C128, V, nrhs, s);
    CKL();
    CK(cudaStreamSynchronize(s));
    if (take_timeouts() > 0) return fail(c, OV_ERR_TIMEOUT, "solve_overlap: a bounded device wait ran out");
    c->info = hist;
    if (st) {
        st->status = status;
        st->outer_iters = outer;
        st->inner_iters = inner_total;
        st->sign_applies = c->sign_count - sign0;
        st->dslash_calls = c->dslash_count - dslash0;
        double worst = 0.0;
        for (int j = 0; j < nrhs; ++j) worst = std::max(worst, res[j]);
        st->true_residual = worst;
        st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != OV_OK) {
        if (c->err.empty() || status == OV_ERR_NOT_CONVERGED)
            fail(c, status, "solve_overlap: status %d after %d outer / %d inner iterations", status, outer, inner_total);
        return status;
    }
    return OV_OK;
}

// Several masses from one right-hand side set (the multi-mass CG of Sec. 3.2).  The first
// defect-correction cycle is shared: its residual is b for every mass (x0 = 0), so one
// multi-shift CG over the chiral sectors of b (undeflated: a shared Krylov space cannot carry a
// per-mass deflation) gives y_i for all masses, and x_i = D(m_i)^+ y_i.  Each mass then finishes
// in solve_impl from x_i (FP64 true residual, deflated cycles).  x: [mass][rhs] ABI spinors.
template <typename R, typename ST = R>
int solve_multi_impl(ov_ctx* c, const std::vector<double>& mass, const SysSet& Srhs, const void* b, void* x,
                     double tol, ov_solve_stats* st, cudaStream_t s) {
    const auto t0 = std::chrono::steady_clock::now();
    const int nrhs = Srhs.n, nm = (int)mass.size(), V = c->g.V;
    const long long n12 = 12LL * V;
    const int prec = prec_of<R>();
    const size_t vb64 = vec_bytes(c, OV_PREC_F64), vb = vec_bytes(c, prec);
    const size_t abi_bytes = (size_t)nrhs * (size_t)n12 * 16;  // complex128 ABI spinors of one mass
    void *B, *S64, *Bs, *Z, *Ysum, *E, *E64;
    TRY(workspace(c, "mm_B", OV_PREC_F64, nrhs, &B));
    TRY(workspace(c, "mm_S64", OV_PREC_F64, 2 * nrhs, &S64));
    TRY(workspace(c, "mm_Bs", prec, 2 * nrhs, &Bs));
    TRY(workspace(c, "mm_Z", prec, (long long)nm * 2 * nrhs, &Z));
    TRY(workspace(c, "mm_Ysum", prec, nrhs, &Ysum));
    TRY(workspace(c, "mm_E", prec, nrhs, &E));
    TRY(workspace(c, "mm_E64", OV_PREC_F64, nrhs, &E64));
    TRY(ensure_small(c, 0, (long long)kRedBlocks * 2 * nrhs, 2 * nrhs));
    launch_pack_spinor<double>(b, OV_C128, B, V, nrhs, s);
    CKL();
    const long long dslash0 = c->dslash_count, sign0 = c->sign_count;
    std::vector<double> bn2(nrhs);
    norm2_rhs<double>(B, n12, nrhs, bn2.data(), c->d_partial, c->d_red, s);
    for (int j = 0; j < nrhs; ++j)
        if (!std::isfinite(bn2[j])) return fail(c, OV_ERR_NAN, "NaN/Inf in b (rhs %d)", j);
    // chiral sectors of b
    std::vector<int> src, sys_of_rhs(2 * nrhs, -1);
    std::vector<signed char> chi;
    for (int j = 0; j < nrhs; ++j)
        if (bn2[j] > 0.0)
            for (int sg = 0; sg < 2; ++sg) {
                src.push_back(j);
                chi.push_back(sg == 0 ? 1 : -1);
            }
    const int ns0 = (int)src.size();
    SysSet S;
    std::vector<double> tol_rel;
    int ns = 0, iters = 0, degree = 0, rc = OV_OK;
    if (ns0 > 0) {
        CK(cudaMemcpyAsync(c->d_idx, src.data(), sizeof(int) * ns0, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->d_chi, chi.data(), ns0, cudaMemcpyHostToDevice, s));
        launch_chiral_split<double>(B, S64, c->d_idx, c->d_chi, V, ns0, s);
        CKL();
        std::vector<double> sn2(ns0);
        norm2_rhs<double>(S64, n12, ns0, sn2.data(), c->d_partial, c->d_red, s);
        const double base_tol = inner_base_tol<R, ST>(c);
        for (int k = 0; k < ns0; ++k) {
            const int j = src[k];
            if (!(sn2[k] > 0.0) || std::sqrt(sn2[k]) <= 0.25 * tol * std::sqrt(bn2[j])) continue;
            if (ns != k)
                CK(cudaMemcpyAsync((char*)S64 + (size_t)ns * vb64, (char*)S64 + (size_t)k * vb64, vb64,
                                   cudaMemcpyDeviceToDevice, s));
            S.phase.push_back(Srhs.phase[j]);
            S.chi.push_back(chi[k]);
            sys_of_rhs[2 * j + (chi[k] > 0 ? 0 : 1)] = ns;
            tol_rel.push_back(std::min(0.5, std::max(base_tol, 0.5 * tol * std::sqrt(bn2[j] / sn2[k]))));
            ++ns;
        }
        S.n = ns;
    }
    if (ns > 0) {
        if (std::is_same<R, double>::value)
            CK(cudaMemcpyAsync(Bs, S64, vb64 * ns, cudaMemcpyDeviceToDevice, s));
        else
            launch_convert<double, float>(S64, Bs, V, ns, s);
        CKL();
        // adaptive order: the rule of solve_impl with the lightest mass, which binds
        if (c->p.adaptive_order) {
            double g = 1.0, mmin = std::fabs(mass[0]);
            for (double t : tol_rel) g = std::min(g, t);
            for (double m : mass) mmin = std::min(mmin, std::fabs(m));
            degree = degree_for_delta(c, 0.5 * mmin * g);
        }
        rc = inner_cg_shifted<R, ST>(c, mass, S, Bs, Z, tol_rel, c->p.max_iter, &iters, s, degree);
        if (rc != OV_OK && rc != OV_ERR_NOT_CONVERGED) return rc;
    }
    // x_i = D(m_i)^+ (y_{i,+} + y_{i,-})
    for (int i = 0; i < nm; ++i) {
        char* xi = (char*)x + (size_t)i * abi_bytes;
        if (ns == 0) {
            CK(cudaMemsetAsync(xi, 0, abi_bytes, s));
            continue;
        }
        CK(cudaMemcpyAsync(c->d_idx, sys_of_rhs.data(), sizeof(int) * 2 * nrhs, cudaMemcpyHostToDevice, s));
        dim3 grid(std::min<long long>((n12 + 255) / 256, 152 * 4), nrhs);
        merge_sectors_k<R><<<grid, 256, 0, s>>>((const typename C2<R>::T*)((char*)Z + (size_t)i * ns * vb), c->d_idx,
                                                (typename C2<R>::T*)Ysum, n12);
        count_launch();
        CKL();
        TRY((overlap_op<R, ST>(c, Ysum, Srhs, mass[i], true, E, s, degree)));
        if (std::is_same<R, double>::value)
            CK(cudaMemcpyAsync(E64, E, vb64 * nrhs, cudaMemcpyDeviceToDevice, s));
        else
            launch_convert<float, double>(E, E64, V, nrhs, s);
        launch_unpack_spinor<double>(E64, xi, OV_C128, V, nrhs, s);
        CKL();
    }
    CK(cudaStreamSynchronize(s));
    const long long shared_sign = c->sign_count - sign0, shared_dslash = c->dslash_count - dslash0;
    const double shared_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    char buf[160];
    snprintf(buf, sizeof(buf), "multi-mass: %d masses, shared cycle n %d, %d inner, %d systems%s", nm,
             degree > 0 ? degree : c->p.poly_degree, iters, ns, rc == OV_OK ? "" : " (not converged)");
    std::string info = buf;
    int status = OV_OK;
    for (int i = 0; i < nm; ++i) {
        ov_solve_stats sti{};
        const int rci = solve_impl<R, ST>(c, mass[i], Srhs, b, (char*)x + (size_t)i * abi_bytes, tol, &sti, s);
        snprintf(buf, sizeof(buf), " || m %g: ", mass[i]);
        info += buf + c->info;
        if (st) {
            st[i] = sti;
            st[i].outer_iters += ns > 0 ? 1 : 0;
            st[i].inner_iters += iters;
            if (i == 0) {
                st[i].sign_applies += shared_sign;
                st[i].dslash_calls += shared_dslash;
                st[i].seconds += shared_s;
            }
        }
        if (rci != OV_OK) {
            if (rci != OV_ERR_NOT_CONVERGED) return rci;
            status = rci;
        }
    }
    c->info = info;
    return status;
}

int solve_dispatch(ov_ctx* c, double mass, const SysSet& S, const void* b, void* x, double tol, ov_solve_stats* st,
                   cudaStream_t s) {
    switch (c->p.inner_precision) {
        case OV_PREC_F64: return solve_impl<double>(c, mass, S, b, x, tol, st, s);
        case OV_PREC_F32: return solve_impl<float>(c, mass, S, b, x, tol, st, s);
        case OV_PREC_F16: return solve_impl<float, H16>(c, mass, S, b, x, tol, st, s);
        default: return solve_impl<float, B16>(c, mass, S, b, x, tol, st, s);
    }
}

}  // namespace

extern "C" int solve_overlap_multimass(ov_ctx* c, int n_mass, const double* masses, const double* phase, const void* b,
                                       void* x, int nrhs, double tol, ov_solve_stats* stats, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    if (n_mass < 1 || n_mass > OV_MAX_MASSES || !masses)
        return fail(c, OV_ERR_ARG, "n_mass = %d outside [1, %d] or no masses", n_mass, OV_MAX_MASSES);
    std::vector<double> m(masses, masses + n_mass);
    for (double v : m)
        if (!std::isfinite(v) || !(std::fabs(v) < 2.0))
            return fail(c, OV_ERR_ARG, "mass %g: each mass must be finite with |m| < 2", v);
    if (!(tol > 0.0)) return fail(c, OV_ERR_ARG, "tol must be > 0");
    TRY(check_ready(c, b, x, nrhs));
    SysSet S = make_sys(nrhs, phase);
    TRY(phase_check(c, S));
    cudaStream_t s = (cudaStream_t)stream;
    switch (c->p.inner_precision) {
        case OV_PREC_F64: return solve_multi_impl<double>(c, m, S, b, x, tol, stats, s);
        case OV_PREC_F32: return solve_multi_impl<float>(c, m, S, b, x, tol, stats, s);
        case OV_PREC_F16: return solve_multi_impl<float, H16>(c, m, S, b, x, tol, stats, s);
        default: return solve_multi_impl<float, B16>(c, m, S, b, x, tol, stats, s);
    }
}

extern "C" int solve_overlap(ov_ctx* c, double mass, const double* phase, const void* b, void* x, int nrhs, double tol,
                             ov_solve_stats* stats, ov_stream_t stream) {
    TRY(check_ready(c, b, x, nrhs));
    if (!(tol > 0.0) || !std::isfinite(mass)) return fail(c, OV_ERR_ARG, "tol must be > 0 and mass finite");
    SysSet S = make_sys(nrhs, phase);
    TRY(phase_check(c, S));
    cudaStream_t s = (cudaStream_t)stream;
    return solve_dispatch(c, mass, S, b, x, tol, stats, s);
}

extern "C" int ov_set_inner_precision(ov_ctx* c, int inner_precision) {
    if (!c) return OV_ERR_ARG;
    TRY(check_inner_precision(c, &c->p, inner_precision));
    c->p.inner_precision = inner_precision;
    return OV_OK;
}

extern "C" int ov_eigensolve_overlap(ov_ctx* c, double phase, int chirality, int n_ev, int krylov, double tol,
                                     int max_restarts, double* theta_out, double* res_out, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    if (!c->gauge_set) return fail(c, OV_ERR_STATE, "no gauge field set (call ov_set_gauge first)");
    if (chirality != 1 && chirality != -1) return fail(c, OV_ERR_ARG, "chirality must be +1 or -1");
    if (n_ev < 1 || n_ev > 256) return fail(c, OV_ERR_ARG, "n_ev = %d outside [1, 256]", n_ev);
    if (!std::isfinite(phase)) return fail(c, OV_ERR_ARG, "non-finite phase");
    const int K = krylov > 0 ? krylov : std::max(3 * n_ev, n_ev + 32);
    if (K < n_ev + 16 || K > 2000) return fail(c, OV_ERR_ARG, "krylov = %d outside [n_ev + 16, 2000]", K);
    if (phase != 0.0 && !find_bank(c, phase))
        return fail(c, OV_ERR_NO_BANK, "no small-space bank registered for phase %.17g", phase);
    cudaStream_t s = (cudaStream_t)stream;
    TRY(lanczos_overlap(c, phase, chirality, n_ev, K, tol > 0.0 ? tol : 1e-4, max_restarts >= 0 ? max_restarts : 50, s));
    TRY(dspace_fp64(c, *find_dspace(c, phase, chirality), s));
    CK(cudaStreamSynchronize(s));
    if (take_timeouts() > 0) return fail(c, OV_ERR_TIMEOUT, "D_ov Lanczos: a bounded device wait ran out");
    const DefSpace* sp = find_dspace(c, phase, chirality);
    for (int i = 0; i < n_ev; ++i) {
        if (theta_out) theta_out[i] = sp->theta[i];
        if (res_out) res_out[i] = sp->res[i];
    }
    return OV_OK;
}

extern "C" int ov_clear_overlap_deflation(ov_ctx* c, double phase, int chirality) {
    if (!c) return OV_ERR_ARG;
    for (auto& sp : c->dspaces)
        if (sp.phase == phase && (chirality == 0 || sp.chi == chirality)) {
            CK(cudaDeviceSynchronize());
            for (void** q : {&sp.W, &sp.AW0, &sp.AWm, &sp.W64, &sp.DW64, &sp.DmW64, &sp.AW64, &sp.AWm64})
                if (*q) {
                    CK(cudaFree(*q));
                    *q = nullptr;
                }
            sp.n = 0;
            sp.mass = -1.0;
            sp.dm_mass = -1.0;
        }
    return OV_OK;
}

// ============================================================================
// Derivatives with respect to the field phase phi = q E (background-field method,
// Sec. 4).  The implemented sign function is F(H) = sum_{low} sign(l_i) P_i +
// sum_{high} q(l_i) P_i; its exact derivative along dH = dH_w/dphi is the
// Daleckii-Krein sum dF = sum_ij F[l_i, l_j] P_i dH P_j, taken here in three blocks:
//   high-high  Pi_perp (dq(H)[dH]) Pi_perp: the tangent of the Clenshaw recurrence
//              (recomputed alongside it, nothing stored);
//   low-low    V M V^+, M_ij = (s_i - s_j)/(l_i - l_j) (V^+ dH V)_ij;
//   low-high   sum_i v_i <u_i, .> + u_i <v_i, .>, u_i = sum_{high j} F[l_i, l_j] P_j dH v_i.
// In the low-high block F[l_i, l_j] = (s_i - q(l_j))/(l_i - l_j) is taken with sign(l_j)
// for q(l_j): the two differ by the polynomial error delta.  Then only pairs of opposite
// sign remain, F = 2/(h(|t_i| + |t_j|)) in units of Q (t = l/h), and
// u_i = (2/h) rho_i(Q^2) Pi_perp (1 - s_i sign)/2 dH v_i with rho_i(x) = 1/(|t_i| + sqrt(x)),
// a Chebyshev polynomial per mode on the interval of the sign function.
// ============================================================================

namespace {

// Y_r = P_r(Q^2) X_r for per-system polynomials P_r = sum_k coef[r][k] T_k(Y), Y = (2 Q^2 -
// (1 + eps))/(1 - eps) on the context's interval [eps, 1] (FP64, same Clenshaw recurrence as
// the sign function; coef: device [ns][n+1]).
int poly_per_system(ov_ctx* c, const void* X, const SysSet& S, const double* d_coef, void* Yout, cudaStream_t s) {
    const int ns = S.n;
    void *bA, *bB, *t;
    TRY(workspace(c, "pp_bA", OV_PREC_F64, ns, &bA));
    TRY(workspace(c, "pp_bB", OV_PREC_F64, ns, &bB));
    TRY(workspace(c, "pp_t", OV_PREC_F64, ns, &t));
    TRY(upload_sys(c, S, s));
    const double* d_phase = any_phase(S) ? c->d_phase : nullptr;
    const int n = c->p.poly_degree;
    const double eps = c->p.eps, h = c->hw_norm, m0 = c->p.m0;
    const double alpha = 4.0 / ((1.0 - eps) * h * h);
    const double beta = -2.0 * (1.0 + eps) / (1.0 - eps);
    // b_n = c_n x: an epilogue-only pass (c_op = 0) that scales per system
    Epilogue e0;
    e0.c_op = 0.0;
    e0.c2 = 1.0;
    e0.v2 = X;
    e0.c2r = d_coef + n;
    e0.c2r_stride = n + 1;
    launch_dslash<double>(c->g, m0, c->U64, X, bA, ns, d_phase, e0, s);
    void *b1 = bA, *b2 = nullptr;
    Epilogue plain;
    for (int k = n - 1; k >= 0; --k) {
        const double hf = (k == 0) ? 0.5 : 1.0;
        launch_dslash<double>(c->g, m0, c->U64, b1, t, ns, d_phase, plain, s);
        Epilogue e;
        e.c_op = alpha * hf;
        e.c1 = beta * hf;
        e.v1 = b1;
        e.c2 = 1.0;
        e.v2 = X;
        e.c2r = d_coef + k;
        e.c2r_stride = n + 1;
        e.c3 = -1.0;
        e.v3 = b2;
        void* o = (k == 0) ? Yout : (b2 ? b2 : bB);
        launch_dslash<double>(c->g, m0, c->U64, t, o, ns, d_phase, e, s);
        b2 = b1;
        b1 = o;
    }
    CKL();
    c->dslash_count += (2LL * n + 1) * ns;
    return OV_OK;
}

// Small dense helpers on device matrices through the host (n x k, row-major double2).
int download(ov_ctx* c, const double2* d, size_t n, std::vector<double2>& h, cudaStream_t s) {
    h.resize(n);
    CK(cudaMemcpyAsync(h.data(), d, sizeof(double2) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return OV_OK;
}

// out_j = alpha X_j + sum_i A_i C[i][j] with C given on the host ([na][nb], row-major).
int combine_host(ov_ctx* c, const void* A, int na, const std::vector<double2>& C, int nb, double alpha, const void* X,
                 void* out, cudaStream_t s) {
    const long long n12 = 12LL * c->g.V;
    TRY(ensure_small(c, (long long)na * nb, 0, 1));
    CK(cudaMemcpyAsync(c->d_C, C.data(), sizeof(double2) * na * nb, cudaMemcpyHostToDevice, s));
    combine<double>(A, n12, na, c->d_C, nb, nb, alpha, X, n12, out, n12, n12, s);
    CKL();
    CK(cudaStreamSynchronize(s));  // d_C is reused by the next call
    return OV_OK;
}

// V^+ X for na bank vectors and nb vectors, to the host ([na][nb], row-major).
int vdotx(ov_ctx* c, const void* A, int na, const void* X, int nb, std::vector<double2>& out, cudaStream_t s) {
    const long long n12 = 12LL * c->g.V;
    TRY(ensure_small(c, (long long)na * nb, (long long)na * nb * 4 * 152, 1));
    multidot<double>(A, n12, na, X, n12, nb, n12, c->d_C, c->d_partial, c->partial_cap, s);
    CKL();
    return download(c, c->d_C, (size_t)na * nb, out, s);
}

// Low-low matrix M and low-high vectors u_i of a bank (FP64).
int prepare_bank_derivative(ov_ctx* c, Bank* b, cudaStream_t s) {
    if (b->dready || b->n == 0) {
        b->dready = true;
        return OV_OK;
    }
    const int N = b->n;
    const double h = c->hw_norm;
    const long long n12 = 12LL * c->g.V;
    const size_t vb = vec_bytes(c, OV_PREC_F64);
    void *dV, *SdV, *Z;
    TRY(workspace(c, "dv_dV", OV_PREC_F64, N, &dV));
    TRY(workspace(c, "dv_SdV", OV_PREC_F64, N, &SdV));
    TRY(workspace(c, "dv_Z", OV_PREC_F64, N, &Z));
    SysSet S;
    S.n = N;
    S.phase.assign(N, b->phase);
    TRY(upload_sys(c, S, s));
    Epilogue plain;
    launch_dslash<double>(c->g, c->p.m0, c->U64, b->V64, dV, N, c->d_phase, plain, s, true);  // dH v_i
    CKL();
    // low-low: M_ij = (s_i - s_j)/(h (t_i - t_j)) K_ij,  K = V^+ dH V
    std::vector<double2> K;
    TRY(vdotx(c, b->V64, N, dV, N, K, s));
    b->M.assign((size_t)N * N, make_double2(0, 0));
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (b->signs[i] == b->signs[j]) continue;
            const double f = (b->signs[i] - b->signs[j]) / (h * (b->theta[i] - b->theta[j]));
            b->M[(size_t)i * N + j] = make_double2(f * K[(size_t)i * N + j].x, f * K[(size_t)i * N + j].y);
        }
    // y_i = Pi_perp (1 - s_i sign)/2 dH v_i
    Epilogue fin;
    fin.c_op = 1.0 / h;
    fin.c1 = 1.0;
    TRY(sign_pipeline<double>(c, dV, S, false, fin, SdV, s));
    std::vector<double> a(N), half(N, 0.5);
    for (int i = 0; i < N; ++i) a[i] = -0.5 * b->signs[i];
    launch_axpby<double>(a.data(), SdV, half.data(), dV, n12, N, s);
    CKL();
    std::vector<double2> C;
    TRY(vdotx(c, b->V64, N, dV, N, C, s));
    for (auto& v : C) v = make_double2(-v.x, -v.y);
    TRY(combine_host(c, b->V64, N, C, N, 1.0, dV, SdV, s));  // SdV <- Pi_perp y
    // z_i = rho_i(Q^2) y_i, rho_i(x) = 1/(|t_i| + sqrt(x)): on the opposite-sign part
    // (|t_i| + |Q|)^{-1} = (|t_i| - s_i Q)^{-1}, and bounded on every other part of the large space
    const int n = c->p.poly_degree;
    std::vector<double> coef((size_t)N * (n + 1));
    for (int i = 0; i < N; ++i)
        host_chebyshev_coeffs_shifted_inverse_root(n, c->p.eps, std::fabs(b->theta[i]), &coef[(size_t)i * (n + 1)]);
    double* d_coef = nullptr;
    if (cudaMalloc(&d_coef, sizeof(double) * coef.size()) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "allocation of per-mode coefficients failed");
    }
    CK(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double) * coef.size(), cudaMemcpyHostToDevice, s));
    const int rc = poly_per_system(c, SdV, S, d_coef, Z, s);
    CK(cudaStreamSynchronize(s));
    cudaFree(d_coef);
    TRY(rc);
    if (cudaMalloc(&b->Uh64, vb * N) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OV_ERR_OOM, "allocation of the bank derivative vectors failed");
    }
    launch_scale<double>(2.0 / h, Z, b->Uh64, n12 * N, s);
    CKL();
    CK(cudaStreamSynchronize(s));
    b->dready = true;
    return OV_OK;
}

// Y = dq(H)[dH] X for the polynomial part q(H) = Q P(Q^2) (no projection), FP64: the tangent
// of the Clenshaw recurrence b_k = c_k x + 2 Y b_{k+1} - b_{k+2} with x fixed:
//   db_k = 2 dY b_{k+1} + 2 Y db_{k+1} - db_{k+2},  2 dY = alpha (dH H + H dH),
// and d(Q p) = (dH p + H dp)/h.
int tangent_poly(ov_ctx* c, const void* X, const SysSet& S, void* Y, cudaStream_t s) {
    const int ns = S.n;
    const long long n12 = 12LL * c->g.V;
    const size_t vb = vec_bytes(c, OV_PREC_F64);
    void *bA, *bB, *dA, *dB, *t, *u, *sv, *r;
    TRY(workspace(c, "tg_bA", OV_PREC_F64, ns, &bA));
    TRY(workspace(c, "tg_bB", OV_PREC_F64, ns, &bB));
    TRY(workspace(c, "tg_dA", OV_PREC_F64, ns, &dA));
    TRY(workspace(c, "tg_dB", OV_PREC_F64, ns, &dB));
    TRY(workspace(c, "tg_t", OV_PREC_F64, ns, &t));
    TRY(workspace(c, "tg_u", OV_PREC_F64, ns, &u));
    TRY(workspace(c, "tg_s", OV_PREC_F64, ns, &sv));
    TRY(workspace(c, "tg_r", OV_PREC_F64, ns, &r));
    TRY(upload_sys(c, S, s));
    const double* d_phase = any_phase(S) ? c->d_phase : nullptr;
    const int n = c->p.poly_degree;
    const double eps = c->p.eps, h = c->hw_norm, m0 = c->p.m0;
    const double alpha = 4.0 / ((1.0 - eps) * h * h);
    const double beta = -2.0 * (1.0 + eps) / (1.0 - eps);
    const void* U = c->U64;
    launch_scale<double>(c->coeffs[n], X, bA, ns * n12, s);
    CK(cudaMemsetAsync(dA, 0, vb * ns, s));
    void *b1 = bA, *b2 = nullptr, *db1 = dA, *db2 = nullptr;
    Epilogue plain, derv;
    for (int k = n - 1; k >= 0; --k) {
        const double hf = (k == 0) ? 0.5 : 1.0;
        launch_dslash<double>(c->g, m0, U, b1, t, ns, d_phase, plain, s);          // t = H b1
        launch_dslash<double>(c->g, m0, U, b1, u, ns, d_phase, derv, s, true);     // u = dH b1
        Epilogue es;
        es.c1 = 1.0;
        es.v1 = u;
        launch_dslash<double>(c->g, m0, U, db1, sv, ns, d_phase, es, s);           // s = H db1 + u
        launch_dslash<double>(c->g, m0, U, t, r, ns, d_phase, derv, s, true);      // r = dH t
        Epilogue eb;
        eb.c_op = alpha * hf;
        eb.c1 = beta * hf;
        eb.v1 = b1;
        eb.c2 = c->coeffs[k];
        eb.v2 = X;
        eb.c3 = -1.0;
        eb.v3 = b2;
        void* ob = b2 ? b2 : bB;
        launch_dslash<double>(c->g, m0, U, t, ob, ns, d_phase, eb, s);             // b_k
        Epilogue ed;
        ed.c_op = alpha * hf;
        ed.c1 = beta * hf;
        ed.v1 = db1;
        ed.c2 = alpha * hf;
        ed.v2 = r;
        ed.c3 = -1.0;
        ed.v3 = db2;
        void* od = db2 ? db2 : dB;
        launch_dslash<double>(c->g, m0, U, sv, od, ns, d_phase, ed, s);            // db_k
        b2 = b1;
        b1 = ob;
        db2 = db1;
        db1 = od;
    }
    CKL();
    c->dslash_count += 6LL * n * ns;
    // Y = (H dp + dH p)/h with p = b1, dp = db1
    Epilogue ep;
    ep.c_op = 1.0 / h;
    launch_dslash<double>(c->g, m0, U, b1, t, ns, d_phase, ep, s, true);           // t = dH p / h
    Epilogue ey;
    ey.c_op = 1.0 / h;
    ey.c1 = 1.0;
    ey.v1 = t;
    launch_dslash<double>(c->g, m0, U, db1, Y, ns, d_phase, ey, s);
    CKL();
    return OV_OK;
}

// out = d sign(H_w)/dphi X (FP64 internal vectors), per run of equal phase.
int dsign_dphi(ov_ctx* c, const void* X, const SysSet& Sall, void* out, cudaStream_t s) {
    const size_t vb = vec_bytes(c, OV_PREC_F64);
    void *Xp, *Yt, *T1;
    TRY(workspace(c, "ds_Xp", OV_PREC_F64, Sall.n, &Xp));
    TRY(workspace(c, "ds_Y", OV_PREC_F64, Sall.n, &Yt));
    TRY(workspace(c, "ds_T", OV_PREC_F64, Sall.n, &T1));
    for (int j0 = 0; j0 < Sall.n;) {
        int j1 = j0 + 1;
        while (j1 < Sall.n && Sall.phase[j1] == Sall.phase[j0]) ++j1;
        const int k = j1 - j0;
        SysSet S;
        S.n = k;
        S.phase.assign(k, Sall.phase[j0]);
        const char* Xj = (const char*)X + (size_t)j0 * vb;
        char* Oj = (char*)out + (size_t)j0 * vb;
        Bank* b = find_bank(c, Sall.phase[j0]);
        if (!b && Sall.phase[j0] != 0.0)
            return fail(c, OV_ERR_NO_BANK, "no small-space bank registered for phase %.17g", Sall.phase[j0]);
        const int N = b ? b->n : 0;
        std::vector<double2> Cv, Du, E;
        if (N > 0) {
            TRY(prepare_bank_derivative(c, b, s));
            TRY(vdotx(c, b->V64, N, Xj, k, Cv, s));   // V^+ X
            TRY(vdotx(c, b->Uh64, N, Xj, k, Du, s));  // U^+ X
            std::vector<double2> Cn(Cv.size());
            for (size_t q = 0; q < Cv.size(); ++q) Cn[q] = make_double2(-Cv[q].x, -Cv[q].y);
            TRY(combine_host(c, b->V64, N, Cn, k, 1.0, Xj, Xp, s));  // Xp = X - V V^+ X
        } else {
            CK(cudaMemcpyAsync(Xp, Xj, vb * k, cudaMemcpyDeviceToDevice, s));
        }
        TRY(tangent_poly(c, Xp, S, Yt, s));
        if (N > 0) {
            TRY(vdotx(c, b->V64, N, Yt, k, E, s));
            // C1 = -V^+ Y + M V^+ X + U^+ X   ([N][k])
            std::vector<double2> C1((size_t)N * k);
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < k; ++j) {
                    double re = -E[(size_t)i * k + j].x + Du[(size_t)i * k + j].x;
                    double im = -E[(size_t)i * k + j].y + Du[(size_t)i * k + j].y;
                    for (int l = 0; l < N; ++l) {
                        const double2 m = b->M[(size_t)i * N + l], x = Cv[(size_t)l * k + j];
                        re += m.x * x.x - m.y * x.y;
                        im += m.x * x.y + m.y * x.x;
                    }
                    C1[(size_t)i * k + j] = make_double2(re, im);
                }
            TRY(combine_host(c, b->V64, N, C1, k, 1.0, Yt, T1, s));  // T1 = Y + V C1
            TRY(combine_host(c, b->Uh64, N, Cv, k, 1.0, T1, Oj, s));  // out = T1 + U V^+ X
        } else {
            CK(cudaMemcpyAsync(Oj, Yt, vb * k, cudaMemcpyDeviceToDevice, s));
        }
        j0 = j1;
    }
    return OV_OK;
}

__global__ void timeslice_scale_k(const double2* __restrict__ in, double2* __restrict__ out, const double* __restrict__ w,
                                  long long seg, int Lt, long long total, int g5) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int t = (int)((i / seg) % Lt);
        const int comp = (int)(i % 12);
        double f = w[t];
        if (g5 && comp >= 6) f = -f;
        const double2 v = in[i];
        out[i] = make_double2(f * v.x, f * v.y);
    }
}

}  // namespace

extern "C" {

int ov_apply_dHdphi(ov_ctx* c, const void* in, void* out, int nrhs, const double* phase, ov_stream_t stream) {
    TRY(check_ready(c, in, out, nrhs));
    cudaStream_t s = (cudaStream_t)stream;
    void *X, *Y;
    TRY(workspace(c, "io_in", OV_PREC_F64, nrhs, &X));
    TRY(workspace(c, "io_out", OV_PREC_F64, nrhs, &Y));
    launch_pack_spinor<double>(in, OV_C128, X, c->g.V, nrhs, s);
    SysSet S = make_sys(nrhs, phase);
    TRY(phase_check(c, S));
    TRY(upload_sys(c, S, s));
    Epilogue e;
    launch_dslash<double>(c->g, c->p.m0, c->U64, X, Y, nrhs, c->d_phase, e, s, true);
    launch_unpack_spinor<double>(Y, out, OV_C128, c->g.V, nrhs, s);
    CKL();
    return OV_OK;
}

int ov_apply_dDdphi(ov_ctx* c, const void* in, void* out, int nrhs, double mass, const double* phase,
                    ov_stream_t stream) {
    TRY(check_ready(c, in, out, nrhs));
    if (!std::isfinite(mass)) return fail(c, OV_ERR_ARG, "mass not finite");
    cudaStream_t s = (cudaStream_t)stream;
    void *X, *Y;
    TRY(workspace(c, "dd_in", OV_PREC_F64, nrhs, &X));
    TRY(workspace(c, "dd_out", OV_PREC_F64, nrhs, &Y));
    launch_pack_spinor<double>(in, OV_C128, X, c->g.V, nrhs, s);
    CKL();
    SysSet S = make_sys(nrhs, phase);
    TRY(phase_check(c, S));
    TRY(dsign_dphi(c, X, S, Y, s));
    // dD(m)/dphi = (1 - m/2) gamma5 dsign/dphi
    launch_gamma5<double>(Y, X, c->g.V, nrhs, s);
    launch_scale<double>(1.0 - 0.5 * mass, X, Y, 12LL * c->g.V * nrhs, s);
    launch_unpack_spinor<double>(Y, out, OV_C128, c->g.V, nrhs, s);
    CKL();
    CK(cudaStreamSynchronize(s));
    return OV_OK;
}

int ov_dcorr_dE(ov_ctx* c, double mass, double charge, double E, const void* S, const void* lam, int nrhs, double tol,
                double* dC, ov_stream_t stream) {
    if (!c) return OV_ERR_ARG;
    if (!c->gauge_set) return fail(c, OV_ERR_STATE, "no gauge field set (call ov_set_gauge first)");
    if (!S || !dC) return fail(c, OV_ERR_ARG, "null S or dC");
    if (nrhs < 1 || nrhs > c->p.max_nrhs)
        return fail(c, OV_ERR_ARG, "nrhs = %d outside [1, max_nrhs = %d]", nrhs, c->p.max_nrhs);
    if (!std::isfinite(mass) || !std::isfinite(charge) || !std::isfinite(E))
        return fail(c, OV_ERR_ARG, "mass, charge and E must be finite");
    if (!lam && !(tol > 0.0)) return fail(c, OV_ERR_ARG, "tol must be > 0 for the tangent solve");
    if (lam == S) return fail(c, OV_ERR_ARG, "lam and S must be different buffers");
    cudaStream_t s = (cudaStream_t)stream;
    const int V = c->g.V, Lt = c->g.L[3];
    const long long n12 = 12LL * V;
    const double phase = charge * E;
    SysSet Sph = make_sys(nrhs, nullptr);
    Sph.phase.assign(nrhs, phase);
    TRY(phase_check(c, Sph));
    // u = dD(m)/dphi S = (1 - m/2) gamma5 dF/dphi S (internal FP64 layout, then ABI)
    void *X, *Y, *U;
    TRY(workspace(c, "dc_X", OV_PREC_F64, nrhs, &X));
    TRY(workspace(c, "dc_Y", OV_PREC_F64, nrhs, &Y));
    TRY(workspace(c, "dc_U", OV_PREC_F64, nrhs, &U));  // ABI complex128 [nrhs][site][4][3]
    launch_pack_spinor<double>(S, OV_C128, X, V, nrhs, s);
    CKL();
    TRY(dsign_dphi(c, X, Sph, Y, s));
    launch_gamma5<double>(Y, X, V, nrhs, s);
    launch_scale<double>(1.0 - 0.5 * mass, X, Y, n12 * nrhs, s);
    launch_unpack_spinor<double>(Y, U, OV_C128, V, nrhs, s);
    CKL();
    const void* left = lam;  // <left, right>_t
    const void* right = U;
    if (!lam) {
        // tangent: dS/dE = -q D(m)^-1 u; w = D(m)^-1 u solved here, then <S, w>_t
        void* Wsol;
        TRY(workspace(c, "dc_W", OV_PREC_F64, nrhs, &Wsol));
        CK(cudaMemsetAsync(Wsol, 0, vec_bytes(c, OV_PREC_F64) * nrhs, s));
        ov_solve_stats st{};
        const int rc = solve_dispatch(c, mass, Sph, U, Wsol, tol, &st, s);
        if (rc != OV_OK) return rc;
        left = S;
        right = Wsol;
    }
    const int nseg = nrhs * Lt;
    const long long seg = 12LL * (V / Lt);  // complex numbers per (rhs, timeslice) in the ABI layout
    TRY(ensure_small(c, 0, (long long)kRedBlocks * nseg, nseg));
    std::vector<double2> ip(nseg);
    dot_rhs<double>(left, right, seg, nseg, ip.data(), c->d_partial, c->d_red, s);
    CKL();
    // dC(t) = 2 Re sum_j <S_j, dS_j/dE>_t = -2 q Re sum_j <S_j, w_j>_t (tangent), or the adjoint
    // form's per-timeslice terms -2 q Re sum_j <lam_j, u_j>_t; dC[Lt] = their sum over t
    double total = 0.0;
    for (int t = 0; t < Lt; ++t) {
        double acc = 0.0;
        for (int j = 0; j < nrhs; ++j) acc += ip[(size_t)j * Lt + t].x;
        dC[t] = -2.0 * charge * acc;
        total += dC[t];
    }
    dC[Lt] = total;
    return OV_OK;
}

int ov_correlator(ov_ctx* c, const void* S, int nrhs, double* C, ov_stream_t stream) {
    if (!c || !S || !C || nrhs < 1) return c ? fail(c, OV_ERR_ARG, "invalid correlator arguments") : OV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int Lt = c->g.L[3];
    const long long seg = 12LL * (c->g.V / Lt);  // complex numbers per (rhs, timeslice)
    TRY(ensure_small(c, 0, (long long)kRedBlocks * nrhs * Lt, nrhs * Lt));
    std::vector<double> n2((size_t)nrhs * Lt);
    norm2_rhs<double>(S, seg, nrhs * Lt, n2.data(), c->d_partial, c->d_red, s);
    CKL();
    for (int t = 0; t < Lt; ++t) {
        double acc = 0.0;
        for (int j = 0; j < nrhs; ++j) acc += n2[(size_t)j * Lt + t];
        C[t] = acc;
    }
    return OV_OK;
}

int ov_timeslice_scale(ov_ctx* c, const void* in, void* out, int nrhs, const double* w, int gamma5,
                       ov_stream_t stream) {
    if (!c || !in || !out || !w || nrhs < 1) return c ? fail(c, OV_ERR_ARG, "invalid arguments") : OV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int Lt = c->g.L[3];
    TRY(ensure_small(c, (Lt + 1) / 2 + 1, 0, 1));
    double* d_w = (double*)c->d_C2;
    CK(cudaMemcpyAsync(d_w, w, sizeof(double) * Lt, cudaMemcpyHostToDevice, s));
    const long long seg = 12LL * (c->g.V / Lt), total = 12LL * c->g.V * nrhs;
    timeslice_scale_k<<<152 * 8, 256, 0, s>>>((const double2*)in, (double2*)out, d_w, seg, Lt, total, gamma5);
    count_launch();
    CKL();
    CK(cudaStreamSynchronize(s));  // d_w is reused
    return OV_OK;
}

int ov_inner(ov_ctx* c, const void* a, const void* b, int nrhs, int per_timeslice, double* out, ov_stream_t stream) {
    if (!c || !a || !b || !out || nrhs < 1) return c ? fail(c, OV_ERR_ARG, "invalid arguments") : OV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nseg = per_timeslice ? nrhs * c->g.L[3] : nrhs;
    const long long seg = per_timeslice ? 12LL * (c->g.V / c->g.L[3]) : 12LL * c->g.V;
    TRY(ensure_small(c, 0, (long long)kRedBlocks * nseg, nseg));
    std::vector<double2> r(nseg);
    dot_rhs<double>(a, b, seg, nseg, r.data(), c->d_partial, c->d_red, s);
    CKL();
    for (int j = 0; j < nseg; ++j) {
        out[2 * j] = r[j].x;
        out[2 * j + 1] = r[j].y;
    }
    return OV_OK;
}

}  // extern "C"
