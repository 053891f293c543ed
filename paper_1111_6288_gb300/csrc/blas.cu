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

// ---- packing -------------------------------------------------------------

template <typename TI, typename R>
__global__ void pack_spinor_k(const TI* __restrict__ abi, typename C2<R>::T* __restrict__ out, int V, int nrhs) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)V * nrhs) return;
    const int r = (int)(idx / V), s = (int)(idx % V);
    const TI* src = abi + ((long long)r * V + s) * 12;
    typename C2<R>::T* dst = out + (long long)r * 12 * V + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        typename C2<R>::T v;
        v.x = (R)src[k].x;
        v.y = (R)src[k].y;
        dst[(long long)k * V] = v;
    }
}

template <typename R, typename TO>
__global__ void unpack_spinor_k(const typename C2<R>::T* __restrict__ in, TO* __restrict__ abi, int V, int nrhs) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)V * nrhs) return;
    const int r = (int)(idx / V), s = (int)(idx % V);
    const typename C2<R>::T* src = in + (long long)r * 12 * V + s;
    TO* dst = abi + ((long long)r * V + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        typename C2<R>::T v = src[(long long)k * V];
        TO o;
        o.x = v.x;
        o.y = v.y;
        dst[k] = o;
    }
}

template <typename TI, typename R>
__global__ void pack_gauge_k(const TI* __restrict__ abi, typename C2<R>::T* __restrict__ out, int V) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4LL * V) return;
    const int mu = (int)(idx / V), s = (int)(idx % V);
    const TI* src = abi + ((long long)mu * V + s) * 9;
    typename C2<R>::T* dst = out + (long long)mu * 9 * V + s;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        typename C2<R>::T v;
        v.x = (R)src[k].x;
        v.y = (R)src[k].y;
        dst[(long long)k * V] = v;
    }
}

template <typename RI, typename RO>
__global__ void convert_k(const typename C2<RI>::T* __restrict__ in, typename C2<RO>::T* __restrict__ out,
                          long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        typename C2<RI>::T v = in[i];
        typename C2<RO>::T o;
        o.x = (RO)v.x;
        o.y = (RO)v.y;
        out[i] = o;
    }
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
__global__ void chiral_split_k(const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y,
                               const int* __restrict__ src, const signed char* __restrict__ chi, int V) {
    const int j = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const long long V12 = 12LL * V;
    const typename C2<R>::T* px = x + (long long)src[j] * V12;
    typename C2<R>::T* py = y + (long long)j * V12;
    const int c = chi[j];
    typename C2<R>::T zero;
    zero.x = 0;
    zero.y = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const bool keep = (k < 6) ? (c > 0) : (c < 0);
        py[(long long)k * V + s] = keep ? px[(long long)k * V + s] : zero;
    }
}

template <typename R>
__global__ void gamma5_k(const typename C2<R>::T* __restrict__ x, typename C2<R>::T* __restrict__ y, int V) {
    const int r = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const long long o = (long long)r * 12 * V;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        typename C2<R>::T v = x[o + (long long)k * V + s];
        if (k >= 6) {
            v.x = -v.x;
            v.y = -v.y;
        }
        y[o + (long long)k * V + s] = v;
    }
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

// out_j = alpha X_j + sum_i A_i C[i][j], up to CJ outputs per launch
constexpr int CJ = 8;
template <typename R>
__global__ void __launch_bounds__(256) combine_k(const typename C2<R>::T* __restrict__ A, long long sA, int na,
                                                 const double2* __restrict__ C, int ldc, int j0, int nj, double alpha,
                                                 const typename C2<R>::T* __restrict__ X, long long sX,
                                                 typename C2<R>::T* __restrict__ out, long long sO, long long n) {
    extern __shared__ double2 shC[];  // [na][CJ]
    for (int q = threadIdx.x; q < na * CJ; q += blockDim.x) {
        const int i = q / CJ, j = q % CJ;
        shC[q] = (j < nj) ? C[(long long)i * ldc + j0 + j] : make_double2(0, 0);
    }
    __syncthreads();
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (long long)gridDim.x * blockDim.x) {
        R accr[CJ], acci[CJ];
#pragma unroll
        for (int j = 0; j < CJ; ++j) accr[j] = acci[j] = 0;
        for (int i = 0; i < na; ++i) {
            typename C2<R>::T a = A[(long long)i * sA + m];
#pragma unroll
            for (int j = 0; j < CJ; ++j) {
                const double2 c = shC[i * CJ + j];
                accr[j] += a.x * (R)c.x - a.y * (R)c.y;
                acci[j] += a.x * (R)c.y + a.y * (R)c.x;
            }
        }
        for (int j = 0; j < nj; ++j) {
            typename C2<R>::T o;
            o.x = accr[j];
            o.y = acci[j];
            if (X) {
                typename C2<R>::T xv = X[(long long)(j0 + j) * sX + m];
                o.x += (R)alpha * xv.x;
                o.y += (R)alpha * xv.y;
            }
            out[(long long)(j0 + j) * sO + m] = o;
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
        pack_spinor_k<double2, R><<<g, 256, 0, s>>>((const double2*)abi, (typename C2<R>::T*)internal, V, nrhs);
    else
        pack_spinor_k<float2, R><<<g, 256, 0, s>>>((const float2*)abi, (typename C2<R>::T*)internal, V, nrhs);
    count_launch();
}

template <typename R>
void launch_unpack_spinor(const void* internal, void* abi, int dtype_out, int V, int nrhs, cudaStream_t s) {
    const long long n = (long long)V * nrhs;
    const int g = (int)((n + 255) / 256);
    if (dtype_out == 0)
        unpack_spinor_k<R, double2><<<g, 256, 0, s>>>((const typename C2<R>::T*)internal, (double2*)abi, V, nrhs);
    else
        unpack_spinor_k<R, float2><<<g, 256, 0, s>>>((const typename C2<R>::T*)internal, (float2*)abi, V, nrhs);
    count_launch();
}

template <typename R>
void launch_pack_gauge(const void* abi, int dtype_in, void* internal, int V, cudaStream_t s) {
    const long long n = 4LL * V;
    const int g = (int)((n + 255) / 256);
    if (dtype_in == 0)
        pack_gauge_k<double2, R><<<g, 256, 0, s>>>((const double2*)abi, (typename C2<R>::T*)internal, V);
    else
        pack_gauge_k<float2, R><<<g, 256, 0, s>>>((const float2*)abi, (typename C2<R>::T*)internal, V);
    count_launch();
}

template <typename RI, typename RO>
void launch_convert(const void* in, void* out, long long n, cudaStream_t s) {
    convert_k<RI, RO><<<grid_for(n, 256), 256, 0, s>>>((const typename C2<RI>::T*)in, (typename C2<RO>::T*)out, n);
    count_launch();
}

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
    chiral_split_k<R><<<grid, 128, 0, s>>>((const typename C2<R>::T*)x, (typename C2<R>::T*)y, src, chi, V);
    count_launch();
}

template <typename R>
void launch_gamma5(const void* x, void* y, int V, int nrhs, cudaStream_t s) {
    dim3 grid((V + 127) / 128, nrhs);
    gamma5_k<R><<<grid, 128, 0, s>>>((const typename C2<R>::T*)x, (typename C2<R>::T*)y, V);
    count_launch();
}

template <typename R>
void multidot(const void* A, long long strideA, int na, const void* B, long long strideB, int nb, long long n,
              double2* d_C, double2* d_partial, long long partial_cap, cudaStream_t s) {
    const int ti = (na + MT - 1) / MT, tj = (nb + MT - 1) / MT;
    // enough chunks to fill the GPU about four times over, bounded by the partial buffer
    long long nchunk = (4LL * 152 + ti * tj - 1) / (ti * tj);
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
    const size_t shm = sizeof(double2) * (size_t)na * CJ;
    for (int j0 = 0; j0 < nb; j0 += CJ) {
        const int nj = (nb - j0 < CJ) ? nb - j0 : CJ;
        combine_k<R><<<grid_for(n, 256, 152 * 8), 256, shm, s>>>(
            (const typename C2<R>::T*)A, strideA, na, d_C, ldc, j0, nj, alpha, (const typename C2<R>::T*)X, strideX,
            (typename C2<R>::T*)out, strideO, n);
        count_launch();
    }
}

#define OVL_INST(R)                                                                                                  \
    template void launch_pack_spinor<R>(const void*, int, void*, int, int, cudaStream_t);                           \
    template void launch_unpack_spinor<R>(const void*, void*, int, int, int, cudaStream_t);                         \
    template void launch_pack_gauge<R>(const void*, int, void*, int, cudaStream_t);                                 \
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
                             void*, long long, long long, cudaStream_t);
OVL_INST(double)
OVL_INST(float)
#undef OVL_INST

template void launch_convert<double, float>(const void*, void*, long long, cudaStream_t);
template void launch_convert<float, double>(const void*, void*, long long, cudaStream_t);
template void launch_convert<double, double>(const void*, void*, long long, cudaStream_t);
template void launch_convert<float, float>(const void*, void*, long long, cudaStream_t);

}  // namespace ovl
