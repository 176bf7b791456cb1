// probe_static.cu -- pic_dft_fold_static: the probe-DFT fold without any
// device allocation.
//
// The handle-based path keeps its phase table in memory it allocates at
// pic_create.  Some callers cannot allocate device memory at all: code whose
// device memory is owned entirely by another allocator (a framework's caching
// pool or a fixed arena budgeted at start-up), and latency-critical loops in
// which cudaMalloc/cudaFree would synchronise the device.  For them this file
// holds the phase table in a fixed file-scope __device__ array that the
// library image carries: every GPU that loads the library holds its 2 MiB
// until the process exits, and no call here allocates anything.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace {

constexpr int STATIC_CHUNK = 64;        // samples folded per fill of the table
constexpr int STATIC_MAX_FREQS = 2048;  // largest nf accepted
constexpr int MAX_DEVICES = 64;

// Phase table exp(+i 2 pi f t_s) for one chunk: [STATIC_CHUNK][STATIC_MAX_FREQS][2].
// Shared by every call on a device; each chunk overwrites the entries it
// reads before reading them, so nothing in it has to start at zero.
static __device__ __align__(256) double g_dft_scratch[STATIC_CHUNK * STATIC_MAX_FREQS * 2];

std::mutex g_setup_mutex;
// Device address of g_dft_scratch per ordinal, with the id of the context it
// was looked up in: after a device reset the primary context (and the
// array's address) is new, so the address is looked up again.
double *g_scratch_addr[MAX_DEVICES];
unsigned long long g_scratch_ctx[MAX_DEVICES];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
std::once_flag g_driver_once;

// Unique id of the calling thread's current context (0 if unknown).
unsigned long long current_ctx_id() {
    std::call_once(g_driver_once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(a);
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(b);
        }
    });
    if (!g_ctx_current || !g_ctx_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&c) != CUDA_SUCCESS || !c || g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

__global__ void k_static_phasor(const double *freq, int nf, double *ph, long long n0, int cnt, double dt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (f >= nf || s >= cnt) return;
    const double t = (double)(n0 + s + 1) * dt;
    double sn, cs;
    sincos(2.0 * 3.141592653589793 * freq[f] * t, &sn, &cs);
    ph[((long long)s * nf + f) * 2] = cs;
    ph[((long long)s * nf + f) * 2 + 1] = sn;
}

__global__ void k_static_fold(const double *samples, const double *ph, double *F, int np, int nf, unsigned mask,
                              int cnt, double dt) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int pc = blockIdx.y;
    const int p = pc / 3, c = pc % 3;
    if (f >= nf || p >= np || !(mask & (1u << c))) return;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < cnt; s++) {
        const double v = samples[((long long)s * np + p) * 3 + c];
        re += v * ph[((long long)s * nf + f) * 2];
        im += v * ph[((long long)s * nf + f) * 2 + 1];
    }
    double *out = F + (((long long)p * 3 + c) * nf + f) * 2;
    out[0] += re * dt;
    out[1] += im * dt;
}

// Device address of the scratch array for the current device, looked up with
// that device current the first time and again whenever the device's context
// has changed (a reset); if the context id cannot be read it is looked up on
// every call.
int scratch_for_current_device(double **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        pic::set_last_error(PIC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    if (dev < 0 || dev >= MAX_DEVICES) {
        pic::set_last_error(PIC_ERR_UNSUPPORTED, "device ordinal %d above %d", dev, MAX_DEVICES - 1);
        return PIC_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_ctx_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dft_scratch);
        if (e != cudaSuccess || !p) {
            pic::set_last_error(PIC_ERR_CUDA, "cudaGetSymbolAddress(g_dft_scratch): %s", cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = current_ctx_id();  // the lookup has made the context current if it was not
    }
    *out = g_scratch_addr[dev];
    return PIC_OK;
}

}  // namespace

extern "C" int pic_dft_fold_static(const double *samples, int64_t count, int np, uint32_t comp_mask,
                                   const double *freq_hz, int nf, int64_t first_step, double dt, double *F,
                                   void *stream) {
    pic::set_last_error(PIC_OK, "%s", "");
    if (count < 0 || np < 0 || nf < 0 || (comp_mask & ~7u) || !(dt > 0.0))
        return pic::set_last_error(PIC_ERR_ARG, "bad arguments to pic_dft_fold_static");
    if (nf > STATIC_MAX_FREQS)
        return pic::set_last_error(PIC_ERR_ARG, "pic_dft_fold_static: nf=%d exceeds the static limit of %d frequencies",
                                   nf, STATIC_MAX_FREQS);
    if (np > 20000) return pic::set_last_error(PIC_ERR_ARG, "pic_dft_fold_static: np=%d above 20000", np);
    if (count == 0 || np == 0 || nf == 0 || comp_mask == 0) return PIC_OK;
    if (!samples || !freq_hz || !F) return pic::set_last_error(PIC_ERR_ARG, "NULL device pointer");
    double *ph = nullptr;
    int rc = scratch_for_current_device(&ph);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blk = 128;
    for (int64_t s0 = 0; s0 < count; s0 += STATIC_CHUNK) {
        const int cnt = (int)((count - s0) < STATIC_CHUNK ? (count - s0) : STATIC_CHUNK);
        k_static_phasor<<<dim3((nf + blk - 1) / blk, cnt), blk, 0, s>>>(freq_hz, nf, ph, first_step + s0, cnt, dt);
        k_static_fold<<<dim3((nf + blk - 1) / blk, np * 3), blk, 0, s>>>(samples + s0 * np * 3, ph, F, np, nf,
                                                                         comp_mask, cnt, dt);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return pic::set_last_error(PIC_ERR_CUDA, "pic_dft_fold_static launch: %s", cudaGetErrorString(e));
    return PIC_OK;
}
