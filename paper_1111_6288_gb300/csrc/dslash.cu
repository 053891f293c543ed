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
// Storage (see ovl_internal.h): FP64 spinors are 12 planes of double2 and links
// 9 planes of double2 per direction; FP32 spinors are 6 planes of float4 (two
// components per 16-byte load) and links keep their first two rows in 3 planes
// of float4, the third row being rebuilt as conj(row0 x row1) (SU(3)).  The
// 16-bit formats (half_store.h) are read into FP32 and computed in FP32.
//
// One thread per (site, rhs); each reads the 8 neighbour spinors, 8 links and
// its own site for the mass term and the epilogue vectors.  Threads of the same
// site and different right-hand sides sit in the same block, so the links they
// share are read from DRAM/L2 once and from L1 after.
#include <cstdint>
#include <type_traits>

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
// a * b + c, one rounding (explicit so that every complex multiply-add is four FMAs)
__device__ __forceinline__ float fmar(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return __fma_rn(a, b, c); }
// a * b + z
template <typename R>
__device__ __forceinline__ Cx<R> cfma(Cx<R> a, Cx<R> b, Cx<R> z) {
    return {fmar(a.re, b.re, fmar(-a.im, b.im, z.re)), fmar(a.re, b.im, fmar(a.im, b.re, z.im))};
}
// conj(a) * b + z
template <typename R>
__device__ __forceinline__ Cx<R> cfmac(Cx<R> a, Cx<R> b, Cx<R> z) {
    return {fmar(a.re, b.re, fmar(a.im, b.im, z.re)), fmar(a.re, b.im, fmar(-a.im, b.re, z.im))};
}
template <typename R>
__device__ __forceinline__ Cx<R> cscale(R s, Cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ Cx<R> cconj(Cx<R> a) { return {a.re, -a.im}; }

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

// Row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1).
__device__ __forceinline__ void third_row(Cx<float> (&u)[3][3]) {
    u[2][0] = cconj(csub(cmul(u[0][1], u[1][2]), cmul(u[0][2], u[1][1])));
    u[2][1] = cconj(csub(cmul(u[0][2], u[1][0]), cmul(u[0][0], u[1][2])));
    u[2][2] = cconj(csub(cmul(u[0][0], u[1][1]), cmul(u[0][1], u[1][0])));
}

// ---- storage policies ------------------------------------------------------

template <typename R> struct IO;

template <> struct IO<double> {
    // spinor: 12 planes of double2, component k = 3 spin + colour
    static __device__ __forceinline__ void load(const void* base, long long V, int s, Cx<double> (&p)[12]) {
        const double2* b = (const double2*)base;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 v = __ldg(b + k * V + s);
            p[k] = {v.x, v.y};
        }
    }
    static __device__ __forceinline__ void load_plain(const void* base, long long V, int s, Cx<double> (&p)[12]) {
        const double2* b = (const double2*)base;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 v = b[k * V + s];
            p[k] = {v.x, v.y};
        }
    }
    static __device__ __forceinline__ void store(void* base, long long V, int s, const Cx<double> (&p)[12]) {
        double2* b = (double2*)base;
#pragma unroll
        for (int k = 0; k < 12; ++k) b[k * V + s] = make_double2(p[k].re, p[k].im);
    }
    // link U_mu(site): 9 planes of double2 per direction
    static __device__ __forceinline__ void link(const void* U, long long V, int mu, int site, Cx<double> (&u)[3][3]) {
        const double2* b = (const double2*)U + (long long)mu * 9 * V;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const double2 v = __ldg(b + (i * 3 + j) * V + site);
                u[i][j] = {v.x, v.y};
            }
    }
    static __host__ __device__ __forceinline__ long long rhs_bytes(long long V) { return 192 * V; }
};

template <> struct IO<float> {
    // spinor: 6 planes of float4 holding components (2p, 2p+1)
    static __device__ __forceinline__ void load(const void* base, long long V, int s, Cx<float> (&p)[12]) {
        const float4* b = (const float4*)base;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v = __ldg(b + q * V + s);
            p[2 * q] = {v.x, v.y};
            p[2 * q + 1] = {v.z, v.w};
        }
    }
    static __device__ __forceinline__ void load_plain(const void* base, long long V, int s, Cx<float> (&p)[12]) {
        const float4* b = (const float4*)base;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v = b[q * V + s];
            p[2 * q] = {v.x, v.y};
            p[2 * q + 1] = {v.z, v.w};
        }
    }
    static __device__ __forceinline__ void store(void* base, long long V, int s, const Cx<float> (&p)[12]) {
        float4* b = (float4*)base;
#pragma unroll
        for (int q = 0; q < 6; ++q)
            b[q * V + s] = make_float4(p[2 * q].re, p[2 * q].im, p[2 * q + 1].re, p[2 * q + 1].im);
    }
    // link: rows 0 and 1 in 3 planes of float4 per direction; row 2 = conj(row0 x row1)
    static __device__ __forceinline__ void link(const void* U, long long V, int mu, int site, Cx<float> (&u)[3][3]) {
        const float4* b = (const float4*)U + (long long)mu * 3 * V;
        const float4 a0 = __ldg(b + site), a1 = __ldg(b + V + site), a2 = __ldg(b + 2 * V + site);
        u[0][0] = {a0.x, a0.y};
        u[0][1] = {a0.z, a0.w};
        u[0][2] = {a1.x, a1.y};
        u[1][0] = {a1.z, a1.w};
        u[1][1] = {a2.x, a2.y};
        u[1][2] = {a2.z, a2.w};
        third_row(u);
    }
    static __host__ __device__ __forceinline__ long long rhs_bytes(long long V) { return 96 * V; }
};

// 16-bit storage: converted to FP32 on load, rounded on store (half_store.h).
template <typename S>
struct IOHalf {
    static __device__ __forceinline__ void load(const void* base, long long V, int s, Cx<float> (&p)[12]) {
        float2 q[12];
        half_load_site<S, true>(base, V, s, q);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = {q[k].x, q[k].y};
    }
    static __device__ __forceinline__ void load_plain(const void* base, long long V, int s, Cx<float> (&p)[12]) {
        float2 q[12];
        half_load_site<S, false>(base, V, s, q);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = {q[k].x, q[k].y};
    }
    static __device__ __forceinline__ void store(void* base, long long V, int s, const Cx<float> (&p)[12]) {
        float2 q[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = make_float2(p[k].re, p[k].im);
        half_store_site<S>(base, V, s, q);
    }
    static __device__ __forceinline__ void link(const void* U, long long V, int mu, int site, Cx<float> (&u)[3][3]) {
        float2 r[6];
        half_load_link<S>(U, V, mu, site, r);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            u[0][j] = {r[j].x, r[j].y};
            u[1][j] = {r[3 + j].x, r[3 + j].y};
        }
        third_row(u);
    }
    static __host__ __device__ __forceinline__ long long rhs_bytes(long long V) { return half_rhs_bytes<S>(V); }
};
template <> struct IO<H16> : IOHalf<H16> {};
template <> struct IO<B16> : IOHalf<B16> {};

template <typename R>
struct Args {
    const void* __restrict__ U;
    const void* __restrict__ in;
    void* out;
    const void* v1;
    const void* v2;
    const void* v3;
    const double* phase;
    const signed char* chi;
    const double* c2r;
    long long c2r_stride;
    R c_op, c1, c2, c3, diag;
    R bcf[4];
    int L[4];
    int stride[4];
    int V;
    int g5;
};

// How a hop's product is scaled: not at all (factor 1, or a boundary sign that the FP64 links
// carry), by a real boundary factor (FP32 links cannot carry a sign: their third row is
// rebuilt from the first two), or by a complex factor (the field phase on x hops).
enum { kNoFac = 0, kRealFac = 1, kCplxFac = 2 };

// Accumulate one hop in direction MU from the neighbour spinor p: forward (FWD) uses
// U_mu(n) psi(n+mu) with (1 - gamma_mu); backward uses U_mu(n-mu)^+ psi(n-mu) with (1 + gamma_mu).
template <typename ST, int MU, bool FWD, int KIND, typename R = typename Arith<ST>::type>
__device__ __forceinline__ void hop(const Args<R>& a, const Cx<R> (&p)[12], int link_site, Cx<R> fac,
                                    Cx<R> (&acc)[12]) {
    constexpr int S = FWD ? 2 : 0;  // forward: h = psi_up - G psi_dn (multiply G by -1)
    using G = GBlock<MU>;
    const long long V = a.V;
    Cx<R> h[2][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if constexpr (G::diag) {
            h[0][c] = cadd(p[0 + c], mulu<G::A + S>(p[6 + c]));
            h[1][c] = cadd(p[3 + c], mulu<G::B + S>(p[9 + c]));
        } else {
            h[0][c] = cadd(p[0 + c], mulu<G::A + S>(p[9 + c]));
            h[1][c] = cadd(p[3 + c], mulu<G::B + S>(p[6 + c]));
        }
    }
    Cx<R> u[3][3];
    IO<ST>::link(a.U, V, MU, link_site, u);
    Cx<R> w[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Cx<R> z;
            if constexpr (FWD) {  // U h
                z = cmul(u[i][0], h[s][0]);
                z = cfma(u[i][1], h[s][1], z);
                z = cfma(u[i][2], h[s][2], z);
            } else {  // U^+ h
                z = cmulc(u[0][i], h[s][0]);
                z = cfmac(u[1][i], h[s][1], z);
                z = cfmac(u[2][i], h[s][2], z);
            }
            if constexpr (KIND == kCplxFac) w[s][i] = cmul(fac, z);
            else if constexpr (KIND == kRealFac) w[s][i] = cscale(fac.re, z);
            else w[s][i] = z;
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

// Staged tile of one right-hand side in shared memory: the planes of the storage format, each
// P sites long (slot = position in the staged rows), in the same element formats as in global
// memory.  FP32: 6 planes of float4; FP16: 3 planes of uint4 and the plane of site scales;
// BF16: 3 planes of uint4.
template <typename ST> struct TileIO;
template <> struct TileIO<float> {
    static constexpr int nplanes = 6;
    static __device__ __forceinline__ int elem_bytes(int) { return 16; }
    static __host__ __device__ __forceinline__ long long rhs_tile_bytes(long long P) { return 96 * P; }
    // plane q of one right-hand side in global memory and in the tile
    static __device__ __forceinline__ const char* plane(const char* rhs, long long V, int q) { return rhs + 16 * V * q; }
    static __device__ __forceinline__ unsigned char* tile_plane(unsigned char* t, int P, int q) { return t + 16LL * P * q; }
    static __device__ __forceinline__ void load(const unsigned char* t, int P, int slot, Cx<float> (&p)[12]) {
        const float4* b = (const float4*)t;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float4 v = b[q * P + slot];
            p[2 * q] = {v.x, v.y};
            p[2 * q + 1] = {v.z, v.w};
        }
    }
};
template <typename S>
struct TileHalf {
    static constexpr int nplanes = HalfSpinor<S>::scaled ? 4 : 3;
    static __device__ __forceinline__ int elem_bytes(int q) { return q < 3 ? 16 : 4; }
    static __host__ __device__ __forceinline__ long long rhs_tile_bytes(long long P) {
        return HalfSpinor<S>::scaled ? 52 * P : 48 * P;
    }
    static __device__ __forceinline__ const char* plane(const char* rhs, long long V, int q) { return rhs + 16 * V * q; }
    static __device__ __forceinline__ unsigned char* tile_plane(unsigned char* t, int P, int q) { return t + 16LL * P * q; }
    static __device__ __forceinline__ void load(const unsigned char* t, int P, int slot, Cx<float> (&p)[12]) {
        float2 v[12];
        half_load_site<S, false>(t, P, slot, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = {v[k].x, v[k].y};
    }
};
template <> struct TileIO<H16> : TileHalf<H16> {};
template <> struct TileIO<B16> : TileHalf<B16> {};

// Where a hop reads its neighbour spinor: global memory by site index, or the staged tile by slot.
template <typename ST>
struct GlobalSrc {
    const void* in;
    long long V;
    template <typename R>
    __device__ __forceinline__ void load(int site, int, Cx<R> (&p)[12]) const { IO<ST>::load(in, V, site, p); }
};
template <typename ST>
struct TileSrc {
    const unsigned char* tile;
    int P;
    template <typename R>
    __device__ __forceinline__ void load(int, int slot, Cx<R> (&p)[12]) const { TileIO<ST>::load(tile, P, slot, p); }
};

// Both hops of direction MU, neighbours read from src (global site index, or tile slots
// slot_f / slot_b).  XCPLX: the x hops carry the complex factor ph (forward) and conj(ph)
// (backward).  FP64 links carry the boundary signs (folded in when they are packed), so FP64
// hops are scaled only by a phase; Dirichlet hops are skipped in both precisions.
template <typename ST, int MU, bool XCPLX, typename SRC, typename R = typename Arith<ST>::type>
__device__ __forceinline__ void both_hops(const Args<R>& a, const SRC& src, int s, int xmu, int slot_f, int slot_b,
                                          Cx<R> ph, Cx<R> (&acc)[12]) {
    constexpr bool FOLD = sizeof(R) == sizeof(double);
    const int L = a.L[MU], st = a.stride[MU];
    Cx<R> p[12];
    // forward neighbour
    {
        const bool edge = xmu == L - 1;
        const int nb = edge ? s - (L - 1) * st : s + st;
        const R f = edge ? a.bcf[MU] : R(1);
        if (f != R(0)) {
            src.load(nb, slot_f, p);
            if constexpr (MU == 0 && XCPLX)
                hop<ST, MU, true, kCplxFac>(a, p, s, FOLD ? ph : Cx<R>{f * ph.re, f * ph.im}, acc);
            else if constexpr (FOLD) hop<ST, MU, true, kNoFac>(a, p, s, {f, R(0)}, acc);
            else hop<ST, MU, true, kRealFac>(a, p, s, {f, R(0)}, acc);
        }
    }
    // backward neighbour
    {
        const bool edge = xmu == 0;
        const int nb = edge ? s + (L - 1) * st : s - st;
        const R f = edge ? a.bcf[MU] : R(1);
        if (f != R(0)) {
            src.load(nb, slot_b, p);
            if constexpr (MU == 0 && XCPLX)
                hop<ST, MU, false, kCplxFac>(a, p, nb, FOLD ? Cx<R>{ph.re, -ph.im} : Cx<R>{f * ph.re, -f * ph.im}, acc);
            else if constexpr (FOLD) hop<ST, MU, false, kNoFac>(a, p, nb, {f, R(0)}, acc);
            else hop<ST, MU, false, kRealFac>(a, p, nb, {f, R(0)}, acc);
        }
    }
}

// exp(i phi_r t) of right-hand side r at time slice t (1 without a field).  The angle is formed
// in FP64 (one multiply); the FP32 kernels take its sine and cosine in FP32 (absolute error
// ~1e-7, below their own rounding), which keeps the slow FP64 pipe of this GPU out of the
// single-precision path.
template <typename R>
__device__ __forceinline__ Cx<R> field_phase(const Args<R>& a, int r, int t) {
    if (!a.phase) return {R(1), R(0)};
    const double ang = a.phase[r] * (double)t;
    if constexpr (sizeof(R) == sizeof(float)) {
        float sn, cs;
        sincosf((float)ang, &sn, &cs);
        return {cs, sn};
    } else {
        double sn, cs;
        sincos(ang, &sn, &cs);
        return {cs, sn};
    }
}

// The epilogue: z = c_op gamma5 (diag psi - acc / 2) (DERIV: c_op gamma5 (-acc / 2)), + c1 v1,
// gamma5, chiral projection, + c2 v2 + c3 v3, stored at site s of right-hand side r.
template <typename ST, bool DERIV, typename R = typename Arith<ST>::type>
__device__ __forceinline__ void finish(const Args<R>& a, int s, int r, const Cx<R> (&psi)[12],
                                       const Cx<R> (&acc)[12]) {
    const long long V = a.V;
    const long long off = (long long)r * IO<ST>::rhs_bytes(V);  // bytes per right-hand side
    const R cop = a.c_op, c1 = a.c1;
    const R c2 = a.c2r ? a.c2 * (R)a.c2r[(long long)r * a.c2r_stride] : a.c2;
    // cd psi + ch acc on the upper spins, negated on the lower
    const R cd = cop * a.diag, ch = R(-0.5) * cop;
    Cx<R> z[12], tmp[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const R sd = k < 6 ? cd : -cd, sh = k < 6 ? ch : -ch;
        if constexpr (DERIV) z[k] = cscale(sh, acc[k]);
        else z[k] = {fmar(sd, psi[k].re, sh * acc[k].re), fmar(sd, psi[k].im, sh * acc[k].im)};
    }
    // + c1 v1
    if (a.v1) {
        IO<ST>::load((const char*)a.v1 + off, V, s, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = cadd(z[k], cscale(c1, tmp[k]));
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
        IO<ST>::load((const char*)a.v2 + off, V, s, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = cadd(z[k], cscale(c2, tmp[k]));
    }
    if (a.v3) {
        // v3 may alias out: plain loads; the same thread reads then writes site s
        IO<ST>::load_plain((const char*)a.v3 + off, V, s, tmp);
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = cadd(z[k], cscale(a.c3, tmp[k]));
    }
    IO<ST>::store((char*)a.out + off, V, s, z);
}

// ---- bulk copies into shared memory (TMA, one dimension) and their barrier ----

__device__ int g_wait_timeouts;  // set by a kernel whose bounded wait ran out
constexpr long long kWaitCycles = 2000000000LL;  // about one second at the SM clock

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bytes (a multiple of 16) from global src to shared dst, both 16-byte aligned; completes on bar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of bar for at most limit cycles; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit = kWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Self-test of the bounded wait: one block waits on an mbarrier that expects bytes no copy will
// bring, for `limit` cycles, then records the timeout exactly as the tiled kernel does.  No copy
// is in flight, so the block returns cleanly.
__global__ void bounded_wait_selftest_k(long long limit) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t bar_a = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(bar_a, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(bar_a, 16u);  // the phase now waits for 16 bytes
    __syncthreads();
    if (!mbar_wait_bounded(bar_a, 0, limit)) {
        if (threadIdx.x == 0) atomicExch(&g_wait_timeouts, 1);
    }
}

// Block = DSLASH_THREADS threads = (DSLASH_THREADS / b sites) x (b right-hand sides), b in
// {1, 2, 4} (the low bits of the caller's launch shape, autotuned by the library; default 1 for one
// right-hand side, else 2), so that the threads of one site share the SM's L1 for the
// site's links.
#ifndef OVL_DSLASH_THREADS
#define OVL_DSLASH_THREADS 128
#endif
#ifndef OVL_DSLASH_MIN_BLOCKS_F32
#define OVL_DSLASH_MIN_BLOCKS_F32 6
#endif
#ifndef OVL_DSLASH_MIN_BLOCKS_F64
#define OVL_DSLASH_MIN_BLOCKS_F64 1
#endif

constexpr int DSLASH_THREADS = OVL_DSLASH_THREADS;

// Blocks per SM that the register allocation must allow.  FP32: 6 (80 registers, no
// spills), 7-9 % faster than the unconstrained 87 registers at 16^3 x 32 and 24^3 x 48,
// where more resident warps hide the latency of the neighbour loads; FP64 needs its
// registers (a cap makes it spill).  The dense FP32 shape (kShapeDense) allows 7 (72
// registers, a few bytes spilled): a grid of up to 7 x 152 blocks then runs in one wave,
// which wins on a 16^3 x 32 lattice with one right-hand side (1024 blocks); the library
// times both shapes per batch size and keeps the faster.
template <typename R> struct MinBlocks;
template <> struct MinBlocks<float> {
    static constexpr int value = OVL_DSLASH_MIN_BLOCKS_F32;
    static constexpr int dense = 7;
};
template <> struct MinBlocks<double> {
    static constexpr int value = OVL_DSLASH_MIN_BLOCKS_F64;
    static constexpr int dense = OVL_DSLASH_MIN_BLOCKS_F64;
};
template <> struct MinBlocks<H16> : MinBlocks<float> {};
template <> struct MinBlocks<B16> : MinBlocks<float> {};

// DERIV: instead of H_w, its derivative with respect to the field phase phi of the
// right-hand side: only the x hops depend on phi, through exp(i phi t) U_x(n) (forward)
// and exp(-i phi t) U_x(n-x)^+ (backward), whose derivatives bring the factors i t and
// -i t; the mass term drops out.
// Hops are accumulated in the order z, t, x, y in every kernel of this file, so that the
// plain and the tiled kernel give the same bits.
template <typename ST, bool DERIV, int MINB>
__global__ void __launch_bounds__(DSLASH_THREADS, MINB) dslash_kernel(Args<typename Arith<ST>::type> a, int nrhs) {
    using R = typename Arith<ST>::type;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (s >= a.V || r >= nrhs) return;
    const long long V = a.V;
    const GlobalSrc<ST> src{(const char*)a.in + (long long)r * IO<ST>::rhs_bytes(V), V};

    int t = s;
    const int x0 = t % a.L[0];
    t /= a.L[0];
    const int x1 = t % a.L[1];
    t /= a.L[1];
    const int x2 = t % a.L[2];
    const int x3 = t / a.L[2];
    const Cx<R> ph = field_phase(a, r, x3);
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    Cx<R> psi[12];
    if constexpr (DERIV) {
        const R tt = (R)x3;
        both_hops<ST, 0, true>(a, src, s, x0, 0, 0, Cx<R>{-tt * ph.im, tt * ph.re}, acc);  // i t exp(i phi t)
    } else {
        both_hops<ST, 2, false>(a, src, s, x2, 0, 0, ph, acc);
        both_hops<ST, 3, false>(a, src, s, x3, 0, 0, ph, acc);
        if (a.phase) both_hops<ST, 0, true>(a, src, s, x0, 0, 0, ph, acc);
        else both_hops<ST, 0, false>(a, src, s, x0, 0, 0, ph, acc);
        both_hops<ST, 1, false>(a, src, s, x1, 0, 0, ph, acc);
        src.load(s, 0, psi);
    }
    finish<ST, DERIV>(a, s, r, psi, acc);
}

// Tiled H_w: a block covers `rows` whole x-rows of one (z, t) slice (blockDim.x = rows * Lx
// sites) for blockDim.y right-hand sides.  At entry one warp stages, per right-hand side and
// plane, the block's rows and the row on each side in y into shared memory with bulk copies
// (TMA) that complete on an mbarrier; meanwhile every thread computes its z and t hops from
// global memory; then the x and y hops and the mass term read the staged rows.  Against the
// plain kernel this removes four of the nine spinor loads per site from L1/L2.  The wait on
// the barrier is bounded: if it runs out the thread records it in g_wait_timeouts, waits once
// more for the copies in flight and returns without writing.
template <typename ST, int MINB>
__global__ void __launch_bounds__(DSLASH_THREADS, MINB) dslash_tiled_kernel(Args<typename Arith<ST>::type> a,
                                                                            int nrhs) {
    using R = typename Arith<ST>::type;
    extern __shared__ __align__(128) unsigned char tiles[];
    __shared__ __align__(8) unsigned long long bar;
    const int L0 = a.L[0], L1 = a.L[1];
    const int T = blockDim.x, rows = T / L0;
    const int P = T + 2 * L0;  // staged sites per plane: the row below, the block's rows, the row above
    const int s0 = blockIdx.x * T;
    const int rbase = blockIdx.y * blockDim.y;
    const int nr = min((int)blockDim.y, nrhs - rbase);
    const int tid = threadIdx.y * T + threadIdx.x;
    const long long V = a.V;
    const long long tile_bytes = TileIO<ST>::rhs_tile_bytes(P);
    const uint32_t bar_a = smem_u32(&bar);
    if (tid == 0) {
        mbar_init(bar_a, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid < 32) {
        const int y0 = (s0 / L0) % L1;
        const int slice0 = s0 - y0 * L0;  // first site of this (z, t) slice
        const int lo = slice0 + ((y0 + L1 - 1) % L1) * L0, hi = slice0 + ((y0 + rows) % L1) * L0;
        constexpr int NP = TileIO<ST>::nplanes;
        if (tid == 0) mbar_expect_tx(bar_a, (uint32_t)(nr * tile_bytes));
        __syncwarp();
        for (int i = tid; i < nr * NP * 3; i += 32) {
            const int seg = i % 3, q = (i / 3) % NP, rr = i / (3 * NP);
            const long long es = TileIO<ST>::elem_bytes(q);
            const char* src = TileIO<ST>::plane((const char*)a.in + (long long)(rbase + rr) * IO<ST>::rhs_bytes(V), V, q);
            unsigned char* dst = TileIO<ST>::tile_plane(tiles + rr * tile_bytes, P, q);
            const int from = seg == 0 ? lo : (seg == 1 ? s0 : hi);
            const int at = seg == 0 ? 0 : (seg == 1 ? L0 : L0 + T);
            const int n = seg == 1 ? T : L0;
            bulk_g2s(smem_u32(dst + at * es), src + from * es, (uint32_t)(n * es), bar_a);
        }
    }
    const int r = rbase + threadIdx.y;
    if (r >= nrhs) return;
    const int s = s0 + threadIdx.x;
    const GlobalSrc<ST> gsrc{(const char*)a.in + (long long)r * IO<ST>::rhs_bytes(V), V};
    int t = s;
    const int x0 = t % L0;
    t /= L0;
    const int x1 = t % L1;
    t /= L1;
    const int x2 = t % a.L[2];
    const int x3 = t / a.L[2];
    const Cx<R> ph = field_phase(a, r, x3);
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    both_hops<ST, 2, false>(a, gsrc, s, x2, 0, 0, ph, acc);
    both_hops<ST, 3, false>(a, gsrc, s, x3, 0, 0, ph, acc);
    if (!mbar_wait_bounded(bar_a, 0)) {
        atomicExch(&g_wait_timeouts, 1);
        mbar_wait_bounded(bar_a, 0);
        return;
    }
    const TileSrc<ST> tsrc{tiles + threadIdx.y * tile_bytes, P};
    const int slot = L0 + threadIdx.x, row0 = slot - x0;  // this site's slot; slot of x = 0 in its row
    const int xf = row0 + (x0 + 1 == L0 ? 0 : x0 + 1), xb = row0 + (x0 == 0 ? L0 - 1 : x0 - 1);
    if (a.phase) both_hops<ST, 0, true>(a, tsrc, s, x0, xf, xb, ph, acc);
    else both_hops<ST, 0, false>(a, tsrc, s, x0, xf, xb, ph, acc);
    both_hops<ST, 1, false>(a, tsrc, s, x1, slot + L0, slot - L0, ph, acc);
    Cx<R> psi[12];
    tsrc.load(s, slot, psi);
    finish<ST, false>(a, s, r, psi, acc);
}

}  // namespace

int tile_rows(const Geom& g, int by) {
    const int L0 = g.L[0], L1 = g.L[1];
    if (L0 % 4 != 0) return 0;  // 16-byte aligned rows of the 4-byte FP16 scale plane
    for (int rows = L1; rows >= 1; --rows)
        if (L1 % rows == 0 && L0 * rows * by <= DSLASH_THREADS && (L0 * rows) % 32 == 0) return rows;
    return 0;
}

void launch_bounded_wait_selftest(long long limit_cycles, cudaStream_t s) {
    bounded_wait_selftest_k<<<1, 32, 0, s>>>(limit_cycles);
    count_launch();
}

int take_wait_timeouts() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(int));
    }
    return v;
}

template <typename S>
void launch_dslash(const Geom& g, double m0, const void* links, const void* in, void* out, int nrhs,
                   const double* d_phase, const Epilogue& e, cudaStream_t s, bool deriv, int shape) {
    using R = typename Arith<S>::type;
    Args<R> a;
    a.U = links;
    a.in = in;
    a.out = out;
    a.v1 = e.v1;
    a.v2 = e.v2;
    a.v3 = e.v3;
    a.phase = d_phase;
    a.chi = e.chi;
    a.c2r = e.c2r;
    a.c2r_stride = e.c2r_stride;
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
    const bool dense = (shape & kShapeDense) != 0;
    int by = (shape & kShapeRhsMask) > 0 ? (shape & kShapeRhsMask) : (nrhs > 1 ? 2 : 1);
    while (by > 1 && by > nrhs) by >>= 1;
    constexpr int mb = MinBlocks<S>::value, md = MinBlocks<S>::dense;
    if constexpr (!std::is_same<S, double>::value) {
        // tiled kernel: whole rows per block, bulk copies need 16-byte aligned planes
        const int rows = (shape & kShapeTiled) && !deriv ? tile_rows(g, by) : 0;
        if (rows > 0 && ((uintptr_t)in & 15) == 0) {
            const int T = g.L[0] * rows;
            dim3 block(T, by), grid(g.V / T, (nrhs + by - 1) / by);
            const size_t smem = (size_t)by * TileIO<S>::rhs_tile_bytes(T + 2 * g.L[0]);
            if (dense) dslash_tiled_kernel<S, md><<<grid, block, smem, s>>>(a, nrhs);
            else dslash_tiled_kernel<S, mb><<<grid, block, smem, s>>>(a, nrhs);
            count_launch();
            return;
        }
    }
    const int bx = DSLASH_THREADS / by;
    dim3 block(bx, by);
    dim3 grid((g.V + bx - 1) / bx, (nrhs + by - 1) / by);
    if constexpr (std::is_same<S, R>::value) {  // the field derivative: FP64 and FP32 storage only
        if (deriv) {
            if (dense) dslash_kernel<S, true, md><<<grid, block, 0, s>>>(a, nrhs);
            else dslash_kernel<S, true, mb><<<grid, block, 0, s>>>(a, nrhs);
            count_launch();
            return;
        }
    }
    if (dense) dslash_kernel<S, false, md><<<grid, block, 0, s>>>(a, nrhs);
    else dslash_kernel<S, false, mb><<<grid, block, 0, s>>>(a, nrhs);
    count_launch();
}

template void launch_dslash<double>(const Geom&, double, const void*, const void*, void*, int, const double*,
                                    const Epilogue&, cudaStream_t, bool, int);
template void launch_dslash<float>(const Geom&, double, const void*, const void*, void*, int, const double*,
                                   const Epilogue&, cudaStream_t, bool, int);
template void launch_dslash<H16>(const Geom&, double, const void*, const void*, void*, int, const double*,
                                 const Epilogue&, cudaStream_t, bool, int);
template void launch_dslash<B16>(const Geom&, double, const void*, const void*, void*, int, const double*,
                                 const Epilogue&, cudaStream_t, bool, int);

}  // namespace ovl
