// Wilson Dirac operator D_w and H_w = gamma5 D_w with a fused epilogue.
//
// Paper, Sec. 2 (eq. 1 and after): H_w = gamma5 D_w; every step of the
// polynomial Q P(Q^2) is an application of H_w, and the Wilson stencil is where
// the overlap operator spends most of its time (Sec. 3.1).  Convention (r = 1):
//
//   D_w psi(n) = (4 + m0) psi(n) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(n) psi(n+mu)
//                                             + (1 + gamma_mu) U_mu(n-mu)^+ psi(n-mu) ]
//
// in the chiral basis gamma_mu = [[0, G_mu], [G_mu^+, 0]] with the 2x2 blocks
// G_x = -i s1, G_y = -i s2, G_z = -i s3, G_t = 1, gamma5 = diag(1, 1, -1, -1).
// (1 -+ gamma_mu) has rank 2: each hop projects the neighbour to a half
// spinor h = psi_up -+ G psi_dn, multiplies h by the link (6 instead of 12
// colour matrix-vector products) and rebuilds the lower half as -+ G^+ (U h).
//
// The background field (Sec. 4) is the phase exp(i phi_j t) on x links, made on
// the fly per right-hand side; boundary factors multiply hops across the edge
// and Dirichlet hops are skipped (no loads).
//
// One thread per (site, rhs); each reads the 8 neighbour spinors, 8 links and
// its own site for the mass term and the epilogue vectors.
#include "ovl_internal.h"

namespace ovl {
namespace {

template <typename R>
struct Cx {
    R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cadd(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> csub(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ Cx<R> cmulc(Cx<R> a, Cx<R> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> cscale(R s, Cx<R> a) { return {s * a.re, s * a.im}; }

// Multiplication by the unit 1, i, -1, -i (code 0..3), resolved at compile time.
template <int CODE, typename R>
__device__ __forceinline__ Cx<R> mulu(Cx<R> z) {
    constexpr int c = ((CODE % 4) + 4) % 4;
    if constexpr (c == 0) return z;
    else if constexpr (c == 1) return {-z.im, z.re};
    else if constexpr (c == 2) return {-z.re, -z.im};
    else return {z.im, -z.re};
}
constexpr int conj_code(int c) { return (4 - c) % 4; }

// Upper-right 2x2 block G of gamma_mu: either diagonal (G00 = A, G11 = B) or
// anti-diagonal (G01 = A, G10 = B), entries as unit codes.
template <int MU> struct GBlock;
template <> struct GBlock<0> { static constexpr bool diag = false; static constexpr int A = 3, B = 3; };  // -i s1
template <> struct GBlock<1> { static constexpr bool diag = false; static constexpr int A = 2, B = 0; };  // -i s2
template <> struct GBlock<2> { static constexpr bool diag = true; static constexpr int A = 3, B = 1; };   // -i s3
template <> struct GBlock<3> { static constexpr bool diag = true; static constexpr int A = 0, B = 0; };   // 1

template <typename R>
__device__ __forceinline__ Cx<R> ld(const typename C2<R>::T* p, long long i) {
    typename C2<R>::T v = __ldg(p + i);
    return {v.x, v.y};
}

template <typename R>
struct Args {
    const typename C2<R>::T* __restrict__ U;
    const typename C2<R>::T* __restrict__ in;
    typename C2<R>::T* out;
    const typename C2<R>::T* v1;
    const typename C2<R>::T* v2;
    const typename C2<R>::T* v3;
    const double* phase;
    const signed char* chi;
    R c_op, c1, c2, c3, diag;
    R bcf[4];
    int L[4];
    int stride[4];
    int V;
    int g5;
};

// Accumulate one hop in direction MU: forward (FWD) uses U_mu(n) psi(n+mu) with
// (1 - gamma_mu); backward uses U_mu(n-mu)^+ psi(n-mu) with (1 + gamma_mu).
template <typename R, int MU, bool FWD>
__device__ __forceinline__ void hop(const Args<R>& a, const typename C2<R>::T* __restrict__ in, int nb, int link_site,
                                    Cx<R> fac, bool complex_fac, Cx<R> (&acc)[12]) {
    constexpr int S = FWD ? 2 : 0;  // forward: h = psi_up - G psi_dn (multiply G by -1)
    using G = GBlock<MU>;
    const long long V = a.V;
    Cx<R> h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Cx<R> p0 = ld<R>(in, 0 * 3 * V + c * V + nb);
        Cx<R> p1 = ld<R>(in, 1 * 3 * V + c * V + nb);
        Cx<R> p2 = ld<R>(in, 2 * 3 * V + c * V + nb);
        Cx<R> p3 = ld<R>(in, 3 * 3 * V + c * V + nb);
        if constexpr (G::diag) {
            h[0][c] = cadd(p0, mulu<G::A + S>(p2));
            h[1][c] = cadd(p1, mulu<G::B + S>(p3));
        } else {
            h[0][c] = cadd(p0, mulu<G::A + S>(p3));
            h[1][c] = cadd(p1, mulu<G::B + S>(p2));
        }
    }
    Cx<R> u[3][3];
    const typename C2<R>::T* Umu = a.U + (long long)MU * 9 * V;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) u[i][j] = ld<R>(Umu, (i * 3 + j) * V + link_site);
    Cx<R> w[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Cx<R> z = {0, 0};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if constexpr (FWD) z = cadd(z, cmul(u[i][j], h[s][j]));   // U h
                else z = cadd(z, cmulc(u[j][i], h[s][j]));               // U^+ h
            }
            w[s][i] = complex_fac ? cmul(fac, z) : cscale(fac.re, z);
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[0 * 3 + c] = cadd(acc[0 * 3 + c], w[0][c]);
        acc[1 * 3 + c] = cadd(acc[1 * 3 + c], w[1][c]);
        // lower half: -+ G^+ w (forward: minus), (G^+)_ab = conj(G_ba)
        if constexpr (G::diag) {
            acc[2 * 3 + c] = cadd(acc[2 * 3 + c], mulu<conj_code(G::A) + S>(w[0][c]));
            acc[3 * 3 + c] = cadd(acc[3 * 3 + c], mulu<conj_code(G::B) + S>(w[1][c]));
        } else {
            acc[2 * 3 + c] = cadd(acc[2 * 3 + c], mulu<conj_code(G::B) + S>(w[1][c]));
            acc[3 * 3 + c] = cadd(acc[3 * 3 + c], mulu<conj_code(G::A) + S>(w[0][c]));
        }
    }
}

template <typename R, int MU>
__device__ __forceinline__ void both_hops(const Args<R>& a, const typename C2<R>::T* __restrict__ in, int s,
                                          const int (&x)[4], Cx<R> ph, Cx<R> (&acc)[12]) {
    const int L = a.L[MU], st = a.stride[MU];
    // forward neighbour
    {
        int nb = (x[MU] == L - 1) ? s - (L - 1) * st : s + st;
        R f = (x[MU] == L - 1) ? a.bcf[MU] : R(1);
        if (f != R(0)) {
            if (MU == 0) hop<R, MU, true>(a, in, nb, s, {f * ph.re, f * ph.im}, true, acc);
            else hop<R, MU, true>(a, in, nb, s, {f, R(0)}, false, acc);
        }
    }
    // backward neighbour
    {
        int nb = (x[MU] == 0) ? s + (L - 1) * st : s - st;
        R f = (x[MU] == 0) ? a.bcf[MU] : R(1);
        if (f != R(0)) {
            if (MU == 0) hop<R, MU, false>(a, in, nb, nb, {f * ph.re, -f * ph.im}, true, acc);
            else hop<R, MU, false>(a, in, nb, nb, {f, R(0)}, false, acc);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(128) dslash_kernel(Args<R> a) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.V) return;
    const int r = blockIdx.y;
    const long long V = a.V;
    const long long off = (long long)r * 12 * V;
    const typename C2<R>::T* __restrict__ in = a.in + off;

    int x[4];
    {
        int t = s;
        x[0] = t % a.L[0]; t /= a.L[0];
        x[1] = t % a.L[1]; t /= a.L[1];
        x[2] = t % a.L[2]; t /= a.L[2];
        x[3] = t;
    }
    Cx<R> ph = {R(1), R(0)};
    if (a.phase) {
        double sn, cs;
        sincos(a.phase[r] * (double)x[3], &sn, &cs);
        ph = {(R)cs, (R)sn};
    }
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    both_hops<R, 0>(a, in, s, x, ph, acc);
    both_hops<R, 1>(a, in, s, x, ph, acc);
    both_hops<R, 2>(a, in, s, x, ph, acc);
    both_hops<R, 3>(a, in, s, x, ph, acc);

    // z = c_op * gamma5 (diag psi - acc/2) + c1 v1
    Cx<R> z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        Cx<R> d = csub(cscale(a.diag, ld<R>(in, k * V + s)), cscale(R(0.5), acc[k]));
        if (k >= 6) d = {-d.re, -d.im};  // gamma5
        z[k] = cscale(a.c_op, d);
    }
    if (a.v1) {
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = cadd(z[k], cscale(a.c1, ld<R>(a.v1 + off, k * V + s)));
    }
    if (a.g5) {
#pragma unroll
        for (int k = 6; k < 12; ++k) z[k] = {-z[k].re, -z[k].im};
    }
    if (a.chi) {
        const int c = a.chi[r];
        if (c > 0) {
#pragma unroll
            for (int k = 6; k < 12; ++k) z[k] = {R(0), R(0)};
        } else if (c < 0) {
#pragma unroll
            for (int k = 0; k < 6; ++k) z[k] = {R(0), R(0)};
#pragma unroll
            for (int k = 6; k < 12; ++k) z[k] = {-z[k].re, -z[k].im};
        }
    }
    if (a.v2) {
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = cadd(z[k], cscale(a.c2, ld<R>(a.v2 + off, k * V + s)));
    }
    if (a.v3) {
        // v3 may alias out: plain loads, same thread reads then writes element (k, s)
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            typename C2<R>::T v = a.v3[off + k * V + s];
            z[k] = cadd(z[k], cscale(a.c3, Cx<R>{v.x, v.y}));
        }
    }
    typename C2<R>::T* out = a.out + off;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        typename C2<R>::T v;
        v.x = z[k].re;
        v.y = z[k].im;
        out[k * V + s] = v;
    }
}

}  // namespace

template <typename R>
void launch_dslash(const Geom& g, double m0, const void* links, const void* in, void* out, int nrhs,
                   const double* d_phase, const Epilogue& e, cudaStream_t s) {
    typedef typename C2<R>::T T;
    Args<R> a;
    a.U = (const T*)links;
    a.in = (const T*)in;
    a.out = (T*)out;
    a.v1 = (const T*)e.v1;
    a.v2 = (const T*)e.v2;
    a.v3 = (const T*)e.v3;
    a.phase = d_phase;
    a.chi = e.chi;
    a.c_op = (R)e.c_op;
    a.c1 = (R)e.c1;
    a.c2 = (R)e.c2;
    a.c3 = (R)e.c3;
    a.diag = (R)(4.0 + m0);
    int st = 1;
    for (int mu = 0; mu < 4; ++mu) {
        a.bcf[mu] = (R)g.bcf[mu];
        a.L[mu] = g.L[mu];
        a.stride[mu] = st;
        st *= g.L[mu];
    }
    a.V = g.V;
    a.g5 = e.g5;
    dim3 block(128);
    dim3 grid((g.V + 127) / 128, nrhs);
    dslash_kernel<R><<<grid, block, 0, s>>>(a);
    count_launch();
}

template void launch_dslash<double>(const Geom&, double, const void*, const void*, void*, int, const double*,
                                    const Epilogue&, cudaStream_t);
template void launch_dslash<float>(const Geom&, double, const void*, const void*, void*, int, const double*,
                                   const Epilogue&, cudaStream_t);

}  // namespace ovl
