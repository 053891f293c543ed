// apply_wilson_noalloc: the Wilson operator for callers that cannot allocate
// device memory.
//
// Some callers may not call cudaMalloc at all: host applications whose memory
// manager owns every device allocation and forbids other allocators, real-time
// loops with a fixed memory budget, and code that must not make the implicit
// device synchronisation that cudaMalloc and cudaFree can cause.  This entry
// point serves them: it takes the gauge field and the spinors in the caller's
// buffers (ABI layouts, complex128) and keeps its packed copies in one
// file-scope device array of fixed size instead of allocating.  The paper has
// no counterpart; it runs the same packing and Wilson kernels as apply_wilson.
//
// The array (OV_NOALLOC_SCRATCH_BYTES, 8 MiB) is loaded with the library and
// held by every GPU that loads it until the process exits.  Its device address
// is looked up with cudaGetSymbolAddress once per device, by the first call on
// that device (with that device current); that first call should therefore
// come before any stream capture.  The field phases travel by value in a kernel
// argument that writes them into the array, so the call reads no host memory
// after it returns.  All calls share the array and it keeps the last call's
// contents: every element a call reads is first written by that same call
// (phases, packed links, packed input, packed output), so nothing needs
// clearing, but calls whose work overlaps on the GPU (different streams, or
// different host threads) race on the array and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/ovl.h"
#include "ovl_internal.h"

namespace {

constexpr size_t kScratchBytes = OV_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

int reject(int code, const char* msg) {
    ovl::set_global_error(msg);
    return code;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// The per-rhs field phases, by value (kMaxRhs doubles = 2 KiB of kernel arguments).
struct PhaseArgs {
    double v[ovl::kMaxRhs];
};

__global__ void store_phases_k(PhaseArgs a, int n, double* __restrict__ out) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) out[j] = a.v[j];
}

// Most sites any call can use (one rhs: 16 (36 V + 24 V) bytes of scratch plus alignment).
constexpr long long kMaxSites = (long long)(kScratchBytes / (sizeof(double2) * 60));

}  // namespace

extern "C" int apply_wilson_noalloc(const int dims[4], const int bc[4], double m0, const void* U, const void* in,
                                    void* out, int nrhs, const double* phase, int hermitian, ov_stream_t stream) {
    if (!dims || !bc || !U || !in || !out) return reject(OV_ERR_ARG, "apply_wilson_noalloc: null argument");
    if (in == out) return reject(OV_ERR_ARG, "apply_wilson_noalloc: in and out must be different buffers");
    if (nrhs < 1 || nrhs > ovl::kMaxRhs) return reject(OV_ERR_ARG, "apply_wilson_noalloc: nrhs out of range");
    if (!std::isfinite(m0)) return reject(OV_ERR_ARG, "apply_wilson_noalloc: m0 not finite");
    ovl::Geom g;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2) return reject(OV_ERR_ARG, "apply_wilson_noalloc: every extent must be >= 2");
        if (bc[mu] < 0 || bc[mu] > 2) return reject(OV_ERR_ARG, "apply_wilson_noalloc: invalid boundary condition");
        g.L[mu] = dims[mu];
        g.bcf[mu] = bc[mu] == OV_BC_PERIODIC ? 1.0 : (bc[mu] == OV_BC_ANTIPERIODIC ? -1.0 : 0.0);
        // bounded before the next product, so that V never overflows: any partial product above
        // the array's capacity already rules the request out
        if (dims[mu] > kMaxSites || V * dims[mu] > kMaxSites) {
            char buf[256];
            snprintf(buf, sizeof(buf),
                     "apply_wilson_noalloc: the lattice has more sites than the fixed %zu bytes of scratch hold "
                     "(at most about %lld sites for one rhs)",
                     kScratchBytes, kMaxSites);
            return reject(OV_ERR_ARG, buf);
        }
        V *= dims[mu];
    }
    if (phase)
        for (int j = 0; j < nrhs; ++j)
            if (!std::isfinite(phase[j])) return reject(OV_ERR_ARG, "apply_wilson_noalloc: non-finite phase");
    // scratch layout: [phases (nrhs doubles)][links 4*9*V][packed in 12*V*nrhs][packed out 12*V*nrhs]
    const size_t c16 = sizeof(double2);
    const size_t b_phase = align256(sizeof(double) * (size_t)nrhs);
    const size_t b_links = align256(c16 * 36 * (size_t)V);
    const size_t b_spin = align256(c16 * 12 * (size_t)V * (size_t)nrhs);
    const size_t need = b_phase + b_links + 2 * b_spin;
    if (need > kScratchBytes) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "apply_wilson_noalloc: %lld sites x %d rhs need %zu bytes of scratch, more than the fixed %zu "
                 "(at most about %lld sites for one rhs)",
                 V, nrhs, need, kScratchBytes, kMaxSites);
        return reject(OV_ERR_ARG, buf);
    }
    g.V = (int)V;
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "apply_wilson_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return reject(OV_ERR_CUDA, buf);
    }
    cudaStream_t s = (cudaStream_t)stream;
    char* p = (char*)base;
    double* d_phase = (double*)p;
    void* links = p + b_phase;
    void* xin = p + b_phase + b_links;
    void* xout = p + b_phase + b_links + b_spin;
    if (phase) {
        PhaseArgs pa;
        for (int j = 0; j < nrhs; ++j) pa.v[j] = phase[j];
        store_phases_k<<<1, 128, 0, s>>>(pa, nrhs, d_phase);
        ovl::count_launch();
    }
    ovl::launch_pack_gauge<double>(U, OV_C128, links, g, s);
    ovl::launch_pack_spinor<double>(in, OV_C128, xin, g.V, nrhs, s);
    ovl::Epilogue ep;
    ep.g5 = hermitian ? 0 : 1;  // gamma5 H_w = D_w
    ovl::launch_dslash<double>(g, m0, links, xin, xout, nrhs, phase ? d_phase : nullptr, ep, s);
    ovl::launch_unpack_spinor<double>(xout, out, OV_C128, g.V, nrhs, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "apply_wilson_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
        return reject(OV_ERR_CUDA, buf);
    }
    return OV_OK;
}
