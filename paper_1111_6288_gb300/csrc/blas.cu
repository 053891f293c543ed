// Layout conversion, vector updates and deterministic reductions.
//
// The vector routines of the overlap solver (Sec. 3.1 names "vector additions
// and scalar products" next to the Wilson stencil): packing between the ABI
// layout and the internal site-major planes, precision conversion, CG updates,
// per-right-hand-side inner products, and the small-space projection
// C = V^+ X, X - V C, V diag(s) C (Sec. 2).
//
// Reductions are deterministic: every block writes a partial sum, and a second
// kernel adds the partials of each output in a fixed order.  Partial sums are
// accumulated in FP64 for FP64 data and in FP32 within a thread for FP32 data,
// then in FP64 across threads and blocks.
#include <algorithm>
#include <type_traits>

#include "ovl_internal.h"

namespace ovl {

std::atomic<long long> g_launches{0};

namespace {

template <typename R>
__device__ __forceinline__ double2 to_d2(typename C2<R>::T v) {
    return make_double2((double)v.x, (double)v.y);
}
template <typename R>
__device__ __forceinline__ typename C2<R>::T from_d2(double2 v) {
    typename C2<R>::T o;
    o.x = (R)v.x;
    o.y = (R)v.y;
    return o;
}

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Block-wide sum of a double2; result valid in thread 0.  Fixed order.
template <int NT>
__device__ double2 block_sum(double2 v) {
    __shared__ double2 sh[NT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double2 r = make_double2(0, 0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) r = dadd(r, sh[i]);
    }
    __syncthreads();
    return r;
}

// ---- per-site spinor access in the internal layouts ------------------------
// FP64: 12 planes of double2; FP32: 6 planes of float4 holding components (2q, 2q+1).
template <typename R> struct SiteIO;
template <> struct SiteIO<double> {
    typedef double2 T;
    static __device__ __forceinline__ void load(const void* b, long long V, long long s, T (&p)[12]) {
        const T* q = (const T*)b;
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = q[k * V + s];
    }
    static __device__ __forceinline__ void store(void* b, long long V, long long s, const T (&p)[12]) {
        T* q = (T*)b;
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k * V + s] = p[k];
    }
};
template <> struct SiteIO<float> {
    typedef float2 T;
    static __device__ __forceinline__ void load(const void* b, long long V, long long s, T (&p)[12]) {
        const float4* q = (const float4*)b;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const float4 v = q[j * V + s];
            p[2 * j] = make_float2(v.x, v.y);
            p[2 * j + 1] = make_float2(v.z, v.w);
        }
    }
    static __device__ __forceinline__ void store(void* b, long long V, long long s, const T (&p)[12]) {
        float4* q = (float4*)b;
#pragma unroll
        for (int j = 0; j < 6; ++j) q[j * V + s] = make_float4(p[2 * j].x, p[2 * j].y, p[2 * j + 1].x, p[2 * j + 1].y);
    }
};

// ---- packing -------------------------------------------------------------

template <typename TI, typename R>
__global__ void pack_spinor_k(const TI* __restrict__ abi, void* __restrict__ out, int V, int nrhs) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)V * nrhs) return;
    const int r = (int)(idx / V), s = (int)(idx % V);
    const TI* src = abi + ((long long)r * V + s) * 12;
    typename SiteIO<R>::T p[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        p[k].x = (R)src[k].x;
        p[k].y = (R)src[k].y;
    }
    SiteIO<R>::store((char*)out + (long long)r * 12 * V * sizeof(typename SiteIO<R>::T), V, s, p);
}

template <typename R, typename TO>
__global__ void unpack_spinor_k(const void* __restrict__ in, TO* __restrict__ abi, int V, int nrhs) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)V * nrhs) return;
    const int r = (int)(idx / V), s = (int)(idx % V);
    typename SiteIO<R>::T p[12];
    SiteIO<R>::load((const char*)in + (long long)r * 12 * V * sizeof(typename SiteIO<R>::T), V, s, p);
    TO* dst = abi + ((long long)r * V + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        TO o;
        o.x = p[k].x;
        o.y = p[k].y;
        dst[k] = o;
    }
}

// FP64 links: 9 planes of double2 per direction, the link U_mu(n) on the last slice of
// direction mu multiplied by that direction's boundary factor when it is -1 (antiperiodic), so
// that the FP64 Wilson kernel needs no boundary multiply (Dirichlet hops are skipped there).
// FP32 links: rows 0 and 1 of U in 3 planes of float4 per direction (entries (0,0)(0,1) |
// (0,2)(1,0) | (1,1)(1,2)); the Wilson kernel rebuilds row 2 = conj(row0 x row1), exact for
// SU(3) links (and so for no link with a sign folded in: FP32 hops apply the factor).
template <typename TI>
__global__ void pack_gauge64_k(const TI* __restrict__ abi, double2* __restrict__ out, Geom g) {
    const int V = g.V;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * V) return;
    const int mu = (int)(idx / V), s = (int)(idx % V);
    int stride = 1;
    for (int nu = 0; nu < mu; ++nu) stride *= g.L[nu];
    const int xmu = (s / stride) % g.L[mu];
    const double f = (xmu == g.L[mu] - 1 && g.bcf[mu] == -1.0) ? -1.0 : 1.0;
    const TI* src = abi + ((long long)mu * V + s) * 9;
    double2* dst = out + (long long)mu * 9 * V + s;
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[(long long)k * V] = make_double2(f * (double)src[k].x, f * (double)src[k].y);
}

template <typename TI>
__global__ void pack_gauge32_k(const TI* __restrict__ abi, float4* __restrict__ out, int V) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * V) return;
    const int mu = (int)(idx / V), s = (int)(idx % V);
    const TI* src = abi + ((long long)mu * V + s) * 9;
    float4* dst = out + (long long)mu * 3 * V + s;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        dst[(long long)q * V] = make_float4((float)src[2 * q].x, (float)src[2 * q].y, (float)src[2 * q + 1].x,
                                            (float)src[2 * q + 1].y);
}

// spinor vectors between precisions (and so between the two internal layouts)
template <typename RI, typename RO>
__global__ void convert_k(const void* __restrict__ in, void* __restrict__ out, int V, long long nvec) {
    const long long total = (long long)V * nvec;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / V, s = i % V;
        typename SiteIO<RI>::T p[12];
        typename SiteIO<RO>::T o[12];
        SiteIO<RI>::load((const char*)in + r * 12 * V * sizeof(typename SiteIO<RI>::T), V, s, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            o[k].x = (RO)p[k].x;
            o[k].y = (RO)p[k].y;
        }
        SiteIO<RO>::store((char*)out + r * 12 * V * sizeof(typename SiteIO<RO>::T), V, s, o);
    }
}

// FP32 spinors -> 16-bit storage (times factor) and back (half_store.h formats).
template <typename S>
__global__ void to_half_k(const void* __restrict__ in, void* __restrict__ out, int V, long long nvec, float factor) {
    const long long total = (long long)V * nvec;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / V, s = i % V;
        float2 p[12];
        SiteIO<float>::load((const char*)in + r * 96 * V, V, s, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = make_float2(factor * p[k].x, factor * p[k].y);
        half_store_site<S>((char*)out + r * half_rhs_bytes<S>(V), V, s, p);
    }
}

template <typename S>
__global__ void from_half_k(const void* __restrict__ in, void* __restrict__ out, int V, long long nvec) {
    const long long total = (long long)V * nvec;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / V, s = i % V;
        float2 p[12];
        half_load_site<S, false>((const char*)in + r * half_rhs_bytes<S>(V), V, s, p);
        SiteIO<float>::store((char*)out + r * 96 * V, V, s, p);
    }
}

// ABI links -> rows 0 and 1 in 16-bit storage.  The boundary factors are applied by the hops.
template <typename TI, typename S>
__global__ void pack_gauge_half_k(const TI* __restrict__ abi, void* __restrict__ out, int V) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * V) return;
    const int mu = (int)(idx / V), s = (int)(idx % V);
    const TI* src = abi + ((long long)mu * V + s) * 9;
    float2 r[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) r[k] = make_float2((float)src[k].x, (float)src[k].y);
    half_store_link<S>(out, V, mu, s, r);
}

// ---- reductions ------------------------------------------------------------

constexpr int RT = 256;

// partial[r][b] = sum over this block's slice of conj(a) b (rhs r)
template <typename R, bool NORM>
__global__ void __launch_bounds__(RT) dot_partial_k(const typename C2<R>::T* __restrict__ a,
                                                    const typename C2<R>::T* __restrict__ b, long long n,
                                                    double2* __restrict__ partial) {
    const int r = blockIdx.y;
    const typename C2<R>::T* pa = a + (long long)r * n;
    const typename C2<R>::T* pb = NORM ? pa : b + (long long)r * n;
    R sre = 0, sim = 0;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        typename C2<R>::T x = pa[i];
        if (NORM) {
            sre += x.x * x.x + x.y * x.y;
        } else {
            typename C2<R>::T y = pb[i];
            sre += x.x * y.x + x.y * y.y;
            sim += x.x * y.y - x.y * y.x;
        }
    }
    double2 tot = block_sum<RT>(make_double2((double)sre, (double)sim));
    if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = tot;
}

// out[r] = sum_b partial[r][b], fixed order
__global__ void __launch_bounds__(RT) sum_partials_k(const double2* __restrict__ partial, int nb,
                                                     double2* __restrict__ out) {
    const int r = blockIdx.x;
    double2 v = make_double2(0, 0);
    for (int i = threadIdx.x; i < nb; i += RT) v = dadd(v, partial[(long long)r * nb + i]);
    double2 tot = block_sum<RT>(v);
    if (threadIdx.x == 0) out[r] = tot;
}

// ---- updates ---------------------------------------------------------------

struct RhsScalars {
    double a[kMaxRhs];
    double b[kMaxRhs];
};

template <typename R>
__global__ void axpby_k(RhsScalars sc, const typename C2<R>::T* __restrict__ x, typename C2<R>::T* y, long long n,
                        int has_x) {
    const int r = blockIdx.y;
    const R a = (R)sc.a[r], b = (R)sc.b[r];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long k = (long long)r * n + i;
        typename C2<R>::T yv = y[k];
        typename C2<R>::T o;
        if (has_x) {
            typename C2<R>::T xv = x[k];
            o.x = a * xv.x + b * yv.x;
            o.y = a * xv.y + b * yv.y;
        } else {
            o.x = b * yv.x;
            o.y = b * yv.y;
        }
        y[k] = o;
    }
}

template <typename R>
__global__ void cg_xr_k(RhsScalars sc, const typename C2<R>::T* __restrict__ p, const typename C2<R>::T* __restrict__ Ap,
                        typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ rr, long long n) {
    const int r = blockIdx.y;
    const R al = (R)sc.a[r];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long k = (long long)r * n + i;
        typename C2<R>::T pv = p[k], av = Ap[k], xv = x[k], rv = rr[k];
        xv.x += al * pv.x;
        xv.y += al * pv.y;
        rv.x -= al * av.x;
        rv.y -= al * av.y;
        x[k] = xv;
        rr[k] = rv;
    }
}

template <typename R>
__global__ void scale_k(R a, const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        typename C2<R>::T v = x[i];
        v.x *= a;
        v.y *= a;
        y[i] = v;
    }
}

// y_j = P_chi_j x_{src_j}: keeps spins 0,1 (chi = +1) or 2,3 (chi = -1).
template <typename R>
__global__ void chiral_split_k(const void* __restrict__ x, void* __restrict__ y, const int* __restrict__ src,
                               const signed char* __restrict__ chi, int V) {
    const int j = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const size_t vb = (size_t)12 * V * sizeof(typename SiteIO<R>::T);
    typename SiteIO<R>::T p[12];
    SiteIO<R>::load((const char*)x + (size_t)src[j] * vb, V, s, p);
    const int c = chi[j];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const bool keep = (k < 6) ? (c > 0) : (c < 0);
        if (!keep) p[k].x = p[k].y = 0;
    }
    SiteIO<R>::store((char*)y + (size_t)j * vb, V, s, p);
}

template <typename R>
__global__ void gamma5_k(const void* __restrict__ x, void* __restrict__ y, int V) {
    const int r = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const size_t vb = (size_t)12 * V * sizeof(typename SiteIO<R>::T);
    typename SiteIO<R>::T p[12];
    SiteIO<R>::load((const char*)x + (size_t)r * vb, V, s, p);
#pragma unroll
    for (int k = 6; k < 12; ++k) {
        p[k].x = -p[k].x;
        p[k].y = -p[k].y;
    }
    SiteIO<R>::store((char*)y + (size_t)r * vb, V, s, p);
}

// ---- multidot (split-K A^+ B) ----------------------------------------------

constexpr int MT = 8;      // vectors per tile, both sides
constexpr int MK = 32;     // elements per slab
constexpr int MNT = 256;   // threads

template <typename R>
__global__ void __launch_bounds__(MNT) multidot_k(const typename C2<R>::T* __restrict__ A, long long sA, int na,
                                                  const typename C2<R>::T* __restrict__ B, long long sB, int nb,
                                                  long long n, long long chunk, double2* __restrict__ partial) {
    __shared__ typename C2<R>::T shA[MT][MK + 1];
    __shared__ typename C2<R>::T shB[MT][MK + 1];
    __shared__ double2 red[MNT];
    const int i0 = blockIdx.y * MT, j0 = blockIdx.z * MT;
    const long long k_begin = (long long)blockIdx.x * chunk;
    const long long k_end = min(n, k_begin + chunk);
    const int t = threadIdx.x;
    const int pair = t & 63, part = t >> 6;  // 64 (i, j) pairs x 4 parts of a slab
    const int pi = pair >> 3, pj = pair & 7;
    R sre = 0, sim = 0;
    for (long long k0 = k_begin; k0 < k_end; k0 += MK) {
        {
            const int v = t >> 5, e = t & 31;  // 8 vectors x 32 elements
            const long long k = k0 + e;
            typename C2<R>::T za, zb;
            za.x = za.y = zb.x = zb.y = 0;
            if (k < k_end) {
                if (i0 + v < na) za = A[(long long)(i0 + v) * sA + k];
                if (j0 + v < nb) zb = B[(long long)(j0 + v) * sB + k];
            }
            shA[v][e] = za;
            shB[v][e] = zb;
        }
        __syncthreads();
#pragma unroll
        for (int e = part * 8; e < part * 8 + 8; ++e) {
            typename C2<R>::T a = shA[pi][e], b = shB[pj][e];
            sre += a.x * b.x + a.y * b.y;
            sim += a.x * b.y - a.y * b.x;
        }
        __syncthreads();
    }
    red[t] = make_double2((double)sre, (double)sim);
    __syncthreads();
    if (t < 64) {
        double2 v = red[t];
        v = dadd(v, red[t + 64]);
        v = dadd(v, red[t + 128]);
        v = dadd(v, red[t + 192]);
        const int i = i0 + (t >> 3), j = j0 + (t & 7);
        if (i < na && j < nb) partial[((long long)blockIdx.x * na + i) * nb + j] = v;
    }
}

__global__ void multidot_sum_k(const double2* __restrict__ partial, int nchunk, int nab, double2* __restrict__ C) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nab) return;
    double2 v = make_double2(0, 0);
    for (int c = 0; c < nchunk; ++c) v = dadd(v, partial[(long long)c * nab + idx]);
    C[idx] = v;
}

// out_j = alpha X_j + sum_i A_i C[i][j], up to CJ outputs per launch; the coefficients are
// converted once to the data precision R in shared memory.
constexpr int CJ = 8;
template <typename R, int CJT>
__global__ void __launch_bounds__(256) combine_k(const typename C2<R>::T* __restrict__ A, long long sA, int na,
                                                 const double2* __restrict__ C, int ldc, int j0, int nj, double alpha,
                                                 const typename C2<R>::T* __restrict__ X, long long sX,
                                                 typename C2<R>::T* __restrict__ out, long long sO, long long n) {
    extern __shared__ unsigned char cmb_raw[];
    typename C2<R>::T* shC = (typename C2<R>::T*)cmb_raw;  // [na][CJT]
    for (int q = threadIdx.x; q < na * CJT; q += blockDim.x) {
        const int i = q / CJT, j = q % CJT;
        const double2 c = (j < nj) ? C[(long long)i * ldc + j0 + j] : make_double2(0, 0);
        shC[q].x = (R)c.x;
        shC[q].y = (R)c.y;
    }
    __syncthreads();
    const R al = (R)alpha;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
        R accr[CJT], acci[CJT];
#pragma unroll
        for (int j = 0; j < CJT; ++j) accr[j] = acci[j] = 0;
        for (int i = 0; i < na; ++i) {
            typename C2<R>::T a = A[(long long)i * sA + m];
#pragma unroll
            for (int j = 0; j < CJT; ++j) {
                const typename C2<R>::T c = shC[i * CJT + j];
                accr[j] += a.x * c.x - a.y * c.y;
                acci[j] += a.x * c.y + a.y * c.x;
            }
        }
        for (int j = 0; j < nj; ++j) {
            typename C2<R>::T o;
            o.x = accr[j];
            o.y = acci[j];
            if (X) {
                typename C2<R>::T xv = X[(long long)(j0 + j) * sX + m];
                o.x += al * xv.x;
                o.y += al * xv.y;
            }
            out[(long long)(j0 + j) * sO + m] = o;
        }
    }
}

// ---- small-space projection for a few right-hand sides ---------------------
//
// C[i][j] = <V_i, X_j> for j < nb <= SP_NB: each warp owns 8 rows of V and walks a
// chunk of the element range, so every element of V is read once; each lane keeps
// 8 x nb partial sums (in R), reduced across the warp in a fixed order and written
// per chunk (the chunks are added by multidot_sum_k, also in a fixed order).
constexpr int SP_NB = 4;
constexpr int SP_ROWS = 8;  // rows per warp; 8 warps -> 64 rows per block

template <typename R, int NB>
__global__ void __launch_bounds__(256) vdot_rows_k(const typename C2<R>::T* __restrict__ V, long long sV, int na,
                                                   const typename C2<R>::T* __restrict__ X, long long sX, int nb,
                                                   long long n, long long chunk, double2* __restrict__ partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.y * 64 + warp * SP_ROWS;
    const long long k_begin = (long long)blockIdx.x * chunk;
    const long long k_end = min(n, k_begin + chunk);
    R ar[SP_ROWS][NB], ai[SP_ROWS][NB];
#pragma unroll
    for (int r = 0; r < SP_ROWS; ++r)
#pragma unroll
        for (int j = 0; j < NB; ++j) ar[r][j] = ai[r][j] = 0;
    for (long long m = k_begin + lane; m < k_end; m += 32) {
        typename C2<R>::T xv[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j < nb) xv[j] = X[(long long)j * sX + m];
            else xv[j].x = xv[j].y = 0;
        }
#pragma unroll
        for (int r = 0; r < SP_ROWS; ++r) {
            const int i = row0 + r;
            if (i < na) {
                const typename C2<R>::T v = V[(long long)i * sV + m];
#pragma unroll
                for (int j = 0; j < NB; ++j) {  // conj(v) * x
                    ar[r][j] += v.x * xv[j].x + v.y * xv[j].y;
                    ai[r][j] += v.x * xv[j].y - v.y * xv[j].x;
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < SP_ROWS; ++r)
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            double re = (double)ar[r][j], im = (double)ai[r][j];
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_down_sync(0xffffffffu, re, o);
                im += __shfl_down_sync(0xffffffffu, im, o);
            }
            const int i = row0 + r;
            if (lane == 0 && i < na && j < nb) partial[((long long)blockIdx.x * na + i) * nb + j] = make_double2(re, im);
        }
}

// Xp_j = X_j - sum_i V_i C[i][j],  Ys_j = sum_i V_i s_i C[i][j]  (j0 <= j < j0 + nj, nj <= SP_NB),
// one pass over V; the coefficients are staged in shared memory in the precision R.
template <typename R, int NB>
__global__ void __launch_bounds__(256) proj_apply_k(const typename C2<R>::T* __restrict__ V, long long sV, int na,
                                                    const double2* __restrict__ C, int ldc, const double* __restrict__ sg,
                                                    int j0, int nj, const typename C2<R>::T* __restrict__ X,
                                                    typename C2<R>::T* __restrict__ Xp, typename C2<R>::T* __restrict__ Ys,
                                                    long long sX, long long n) {
    extern __shared__ unsigned char sp_raw[];
    typename C2<R>::T* cn = (typename C2<R>::T*)sp_raw;  // [na][NB]  -C
    typename C2<R>::T* cs = cn + (size_t)na * NB;     // [na][NB]  s C
    for (int q = threadIdx.x; q < na * NB; q += blockDim.x) {
        const int i = q / NB, j = q % NB;
        const double2 c = (j < nj) ? C[(long long)i * ldc + j0 + j] : make_double2(0, 0);
        cn[q].x = (R)(-c.x);
        cn[q].y = (R)(-c.y);
        cs[q].x = (R)(sg[i] * c.x);
        cs[q].y = (R)(sg[i] * c.y);
    }
    __syncthreads();
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
        R a1r[NB], a1i[NB], a2r[NB], a2i[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) a1r[j] = a1i[j] = a2r[j] = a2i[j] = 0;
        for (int i = 0; i < na; ++i) {
            const typename C2<R>::T v = V[(long long)i * sV + m];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                const typename C2<R>::T c1 = cn[i * NB + j], c2 = cs[i * NB + j];
                a1r[j] += v.x * c1.x - v.y * c1.y;
                a1i[j] += v.x * c1.y + v.y * c1.x;
                a2r[j] += v.x * c2.x - v.y * c2.y;
                a2i[j] += v.x * c2.y + v.y * c2.x;
            }
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j < nj) {
                const long long o = (long long)(j0 + j) * sX + m;
                typename C2<R>::T xv = X[o], p, y;
                p.x = xv.x + a1r[j];
                p.y = xv.y + a1i[j];
                y.x = a2r[j];
                y.y = a2i[j];
                Xp[o] = p;
                Ys[o] = y;
            }
        }
    }
}

inline int grid_for(long long n, int bs, int cap = 152 * 16) {
    long long g = (n + bs - 1) / bs;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// ---- launchers -------------------------------------------------------------

template <typename R>
void launch_pack_spinor(const void* abi, int dtype_in, void* internal, int V, int nrhs, cudaStream_t s) {
    const long long n = (long long)V * nrhs;
    const int g = (int)((n + 255) / 256);
    if (dtype_in == 0)
        pack_spinor_k<double2, R><<<g, 256, 0, s>>>((const double2*)abi, internal, V, nrhs);
    else
        pack_spinor_k<float2, R><<<g, 256, 0, s>>>((const float2*)abi, internal, V, nrhs);
    count_launch();
}

template <typename R>
void launch_unpack_spinor(const void* internal, void* abi, int dtype_out, int V, int nrhs, cudaStream_t s) {
    const long long n = (long long)V * nrhs;
    const int g = (int)((n + 255) / 256);
    if (dtype_out == 0)
        unpack_spinor_k<R, double2><<<g, 256, 0, s>>>(internal, (double2*)abi, V, nrhs);
    else
        unpack_spinor_k<R, float2><<<g, 256, 0, s>>>(internal, (float2*)abi, V, nrhs);
    count_launch();
}

template <typename R>
void launch_pack_gauge(const void* abi, int dtype_in, void* internal, const Geom& geom, cudaStream_t s) {
    const int V = geom.V;
    const long long n = 4LL * V;
    const int g = (int)((n + 255) / 256);
    if (std::is_same<R, double>::value) {
        if (dtype_in == 0) pack_gauge64_k<double2><<<g, 256, 0, s>>>((const double2*)abi, (double2*)internal, geom);
        else pack_gauge64_k<float2><<<g, 256, 0, s>>>((const float2*)abi, (double2*)internal, geom);
    } else {
        if (dtype_in == 0) pack_gauge32_k<double2><<<g, 256, 0, s>>>((const double2*)abi, (float4*)internal, V);
        else pack_gauge32_k<float2><<<g, 256, 0, s>>>((const float2*)abi, (float4*)internal, V);
    }
    count_launch();
}

template <typename RI, typename RO>
void launch_convert(const void* in, void* out, int V, long long nvec, cudaStream_t s) {
    convert_k<RI, RO><<<grid_for((long long)V * nvec, 256), 256, 0, s>>>(in, out, V, nvec);
    count_launch();
}

template <typename S>
void launch_to_half(const void* in32, void* out, int V, long long nvec, double factor, cudaStream_t s) {
    to_half_k<S><<<grid_for((long long)V * nvec, 256), 256, 0, s>>>(in32, out, V, nvec, (float)factor);
    count_launch();
}

template <typename S>
void launch_from_half(const void* in, void* out32, int V, long long nvec, cudaStream_t s) {
    from_half_k<S><<<grid_for((long long)V * nvec, 256), 256, 0, s>>>(in, out32, V, nvec);
    count_launch();
}

template <typename S>
void launch_pack_gauge_half(const void* abi, int dtype_in, void* internal, int V, cudaStream_t s) {
    const int g = (int)((4LL * V + 255) / 256);
    if (dtype_in == 0) pack_gauge_half_k<double2, S><<<g, 256, 0, s>>>((const double2*)abi, internal, V);
    else pack_gauge_half_k<float2, S><<<g, 256, 0, s>>>((const float2*)abi, internal, V);
    count_launch();
}

template void launch_to_half<H16>(const void*, void*, int, long long, double, cudaStream_t);
template void launch_to_half<B16>(const void*, void*, int, long long, double, cudaStream_t);
template void launch_from_half<H16>(const void*, void*, int, long long, cudaStream_t);
template void launch_from_half<B16>(const void*, void*, int, long long, cudaStream_t);
template void launch_pack_gauge_half<H16>(const void*, int, void*, int, cudaStream_t);
template void launch_pack_gauge_half<B16>(const void*, int, void*, int, cudaStream_t);

template <typename R>
void dot_rhs(const void* a, const void* b, long long n, int nrhs, double2* host_out, double2* d_partial,
             double2* d_out, cudaStream_t s) {
    dim3 grid(kRedBlocks, nrhs);
    dot_partial_k<R, false><<<grid, RT, 0, s>>>((const typename C2<R>::T*)a, (const typename C2<R>::T*)b, n, d_partial);
    count_launch();
    sum_partials_k<<<nrhs, RT, 0, s>>>(d_partial, kRedBlocks, d_out);
    count_launch();
    cudaMemcpyAsync(host_out, d_out, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
}

template <typename R>
void norm2_rhs(const void* a, long long n, int nrhs, double* host_out, double2* d_partial, double2* d_out,
               cudaStream_t s) {
    dim3 grid(kRedBlocks, nrhs);
    dot_partial_k<R, true><<<grid, RT, 0, s>>>((const typename C2<R>::T*)a, nullptr, n, d_partial);
    count_launch();
    sum_partials_k<<<nrhs, RT, 0, s>>>(d_partial, kRedBlocks, d_out);
    count_launch();
    std::vector<double2> tmp(nrhs);
    cudaMemcpyAsync(tmp.data(), d_out, sizeof(double2) * nrhs, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    for (int r = 0; r < nrhs; ++r) host_out[r] = tmp[r].x;
}

template <typename R>
void launch_axpby(const double* a, const void* x, const double* b, void* y, long long n, int nrhs, cudaStream_t s) {
    RhsScalars sc;
    for (int r = 0; r < nrhs; ++r) {
        sc.a[r] = a ? a[r] : 0.0;
        sc.b[r] = b[r];
    }
    dim3 grid(grid_for(n, 256, 152 * 4), nrhs);
    axpby_k<R><<<grid, 256, 0, s>>>(sc, (const typename C2<R>::T*)x, (typename C2<R>::T*)y, n, x != nullptr);
    count_launch();
}

template <typename R>
void launch_cg_xr(const double* alpha, const void* p, const void* Ap, void* x, void* r, long long n, int nrhs,
                  cudaStream_t s) {
    RhsScalars sc;
    for (int j = 0; j < nrhs; ++j) sc.a[j] = alpha[j];
    dim3 grid(grid_for(n, 256, 152 * 4), nrhs);
    cg_xr_k<R><<<grid, 256, 0, s>>>(sc, (const typename C2<R>::T*)p, (const typename C2<R>::T*)Ap,
                                    (typename C2<R>::T*)x, (typename C2<R>::T*)r, n);
    count_launch();
}

template <typename R>
void launch_scale(double a, const void* x, void* y, long long n, cudaStream_t s) {
    scale_k<R><<<grid_for(n, 256), 256, 0, s>>>((R)a, (const typename C2<R>::T*)x, (typename C2<R>::T*)y, n);
    count_launch();
}

template <typename R>
void launch_chiral_split(const void* x, void* y, const int* src, const signed char* chi, int V, int nsys,
                         cudaStream_t s) {
    dim3 grid((V + 127) / 128, nsys);
    chiral_split_k<R><<<grid, 128, 0, s>>>(x, y, src, chi, V);
    count_launch();
}

template <typename R>
void launch_gamma5(const void* x, void* y, int V, int nrhs, cudaStream_t s) {
    dim3 grid((V + 127) / 128, nrhs);
    gamma5_k<R><<<grid, 128, 0, s>>>(x, y, V);
    count_launch();
}

// C = A^+ B for nb <= NB columns through the row-dot kernel of the small-space projection (chunks of
// at most 4096 elements, so that each lane's FP32 partial sum stays short).
template <typename R, int NB>
void multidot_few(const void* A, long long sA, int na, const void* B, long long sB, int nb, long long n, double2* d_C,
                  double2* d_partial, long long partial_cap, cudaStream_t s) {
    typedef typename C2<R>::T T;
    const int rowblocks = (na + 63) / 64;
    long long nchunk = std::max((4LL * 152 + rowblocks - 1) / rowblocks, (n + 4095) / 4096);
    const long long cap = partial_cap / ((long long)na * nb);
    if (nchunk > cap) nchunk = std::max(1LL, cap);
    long long chunk = (n + nchunk - 1) / nchunk;
    chunk = ((chunk + 31) / 32) * 32;
    nchunk = (n + chunk - 1) / chunk;
    dim3 grid((unsigned)nchunk, rowblocks);
    vdot_rows_k<R, NB><<<grid, 256, 0, s>>>((const T*)A, sA, na, (const T*)B, sB, nb, n, chunk, d_partial);
    count_launch();
    const int nab = na * nb;
    multidot_sum_k<<<(nab + 255) / 256, 256, 0, s>>>(d_partial, (int)nchunk, nab, d_C);
    count_launch();
}

template <typename R>
void multidot(const void* A, long long strideA, int na, const void* B, long long strideB, int nb, long long n,
              double2* d_C, double2* d_partial, long long partial_cap, cudaStream_t s) {
    if (nb <= 4) {  // few columns: one warp per 8 rows, every element of A read once, no padded pairs
        if (nb == 1) multidot_few<R, 1>(A, strideA, na, B, strideB, nb, n, d_C, d_partial, partial_cap, s);
        else if (nb == 2) multidot_few<R, 2>(A, strideA, na, B, strideB, nb, n, d_C, d_partial, partial_cap, s);
        else multidot_few<R, 4>(A, strideA, na, B, strideB, nb, n, d_C, d_partial, partial_cap, s);
        return;
    }
    const int ti = (na + MT - 1) / MT, tj = (nb + MT - 1) / MT;
    // enough chunks to fill the GPU about four times over, bounded by the partial buffer
    // enough chunks to fill the GPU, and chunks of at most 4096 elements (each thread's partial
    // sum then covers about 1000 products, short enough for FP32 accumulation)
    long long nchunk = std::max((4LL * 152 + ti * tj - 1) / (ti * tj), (n + 4095) / 4096);
    const long long max_chunk_by_cap = partial_cap / ((long long)na * nb);
    if (nchunk > max_chunk_by_cap) nchunk = max_chunk_by_cap;
    if (nchunk < 1) nchunk = 1;
    long long chunk = (n + nchunk - 1) / nchunk;
    chunk = ((chunk + MK - 1) / MK) * MK;
    nchunk = (n + chunk - 1) / chunk;
    dim3 grid((unsigned)nchunk, ti, tj);
    multidot_k<R><<<grid, MNT, 0, s>>>((const typename C2<R>::T*)A, strideA, na, (const typename C2<R>::T*)B, strideB,
                                       nb, n, chunk, d_partial);
    count_launch();
    const int nab = na * nb;
    multidot_sum_k<<<(nab + 255) / 256, 256, 0, s>>>(d_partial, (int)nchunk, nab, d_C);
    count_launch();
}

template <typename R>
void combine(const void* A, long long strideA, int na, const double2* d_C, int ldc, int nb, double alpha,
             const void* X, long long strideX, void* out, long long strideO, long long n, cudaStream_t s) {
    if (nb == 1) {  // one column: no padding columns in the inner loop
        const size_t shm1 = sizeof(typename C2<R>::T) * (size_t)na;
        combine_k<R, 1><<<grid_for(n, 256, 152 * 8), 256, shm1, s>>>(
            (const typename C2<R>::T*)A, strideA, na, d_C, ldc, 0, 1, alpha, (const typename C2<R>::T*)X, strideX,
            (typename C2<R>::T*)out, strideO, n);
        count_launch();
        return;
    }
    const size_t shm = sizeof(typename C2<R>::T) * (size_t)na * CJ;
    for (int j0 = 0; j0 < nb; j0 += CJ) {
        const int nj = (nb - j0 < CJ) ? nb - j0 : CJ;
        combine_k<R, CJ><<<grid_for(n, 256, 152 * 8), 256, shm, s>>>(
            (const typename C2<R>::T*)A, strideA, na, d_C, ldc, j0, nj, alpha, (const typename C2<R>::T*)X, strideX,
            (typename C2<R>::T*)out, strideO, n);
        count_launch();
    }
}

template <typename R, int NB>
void small_space_group(const void* V, int na, const double* d_signs, const void* X, int j0, int nj, void* Xp, void* Ys,
                       long long n, double2* d_C, double2* d_partial, long long partial_cap, cudaStream_t s) {
    typedef typename C2<R>::T T;
    const int rowblocks = (na + 63) / 64;
    long long nchunk = std::max(1LL, (4LL * 152) / rowblocks);
    const long long cap = partial_cap / ((long long)na * nj);
    if (nchunk > cap) nchunk = std::max(1LL, cap);
    long long chunk = (n + nchunk - 1) / nchunk;
    chunk = ((chunk + 31) / 32) * 32;
    nchunk = (n + chunk - 1) / chunk;
    dim3 grid((unsigned)nchunk, rowblocks);
    vdot_rows_k<R, NB><<<grid, 256, 0, s>>>((const T*)V, n, na, (const T*)X + (long long)j0 * n, n, nj, n, chunk,
                                            d_partial);
    count_launch();
    const int nab = na * nj;
    multidot_sum_k<<<(nab + 255) / 256, 256, 0, s>>>(d_partial, (int)nchunk, nab, d_C);
    count_launch();
    const size_t shm = 2 * sizeof(T) * (size_t)na * NB;
    proj_apply_k<R, NB><<<grid_for(n, 256, 152 * 8), 256, shm, s>>>((const T*)V, n, na, d_C, nj, d_signs, 0, nj,
                                                                    (const T*)X + (long long)j0 * n,
                                                                    (T*)Xp + (long long)j0 * n,
                                                                    (T*)Ys + (long long)j0 * n, n, n);
    count_launch();
}

template <typename R>
void small_space_project(const void* V, int na, const double* d_signs, const void* X, int nb, void* Xp, void* Ys,
                         long long n, double2* d_C, double2* d_partial, long long partial_cap, cudaStream_t s) {
    for (int j0 = 0; j0 < nb; j0 += SP_NB) {
        const int nj = std::min(SP_NB, nb - j0);
        if (nj == 1) small_space_group<R, 1>(V, na, d_signs, X, j0, nj, Xp, Ys, n, d_C, d_partial, partial_cap, s);
        else if (nj == 2) small_space_group<R, 2>(V, na, d_signs, X, j0, nj, Xp, Ys, n, d_C, d_partial, partial_cap, s);
        else small_space_group<R, 4>(V, na, d_signs, X, j0, nj, Xp, Ys, n, d_C, d_partial, partial_cap, s);
    }
}

#define OVL_INST(R)                                                                                                  \
    template void launch_pack_spinor<R>(const void*, int, void*, int, int, cudaStream_t);                           \
    template void launch_unpack_spinor<R>(const void*, void*, int, int, int, cudaStream_t);                         \
    template void launch_pack_gauge<R>(const void*, int, void*, const Geom&, cudaStream_t);                                 \
    template void dot_rhs<R>(const void*, const void*, long long, int, double2*, double2*, double2*, cudaStream_t); \
    template void norm2_rhs<R>(const void*, long long, int, double*, double2*, double2*, cudaStream_t);             \
    template void launch_axpby<R>(const double*, const void*, const double*, void*, long long, int, cudaStream_t);  \
    template void launch_cg_xr<R>(const double*, const void*, const void*, void*, void*, long long, int,            \
                                  cudaStream_t);                                                                   \
    template void launch_scale<R>(double, const void*, void*, long long, cudaStream_t);                             \
    template void launch_chiral_split<R>(const void*, void*, const int*, const signed char*, int, int,              \
                                         cudaStream_t);                                                            \
    template void launch_gamma5<R>(const void*, void*, int, int, cudaStream_t);                                     \
    template void multidot<R>(const void*, long long, int, const void*, long long, int, long long, double2*,        \
                              double2*, long long, cudaStream_t);                                                  \
    template void combine<R>(const void*, long long, int, const double2*, int, int, double, const void*, long long, \
                             void*, long long, long long, cudaStream_t);                                           \
    template void small_space_project<R>(const void*, int, const double*, const void*, int, void*, void*, long long, \
                                         double2*, double2*, long long, cudaStream_t);
OVL_INST(double)
OVL_INST(float)
#undef OVL_INST

template void launch_convert<double, float>(const void*, void*, int, long long, cudaStream_t);
template void launch_convert<float, double>(const void*, void*, int, long long, cudaStream_t);

}  // namespace ovl
