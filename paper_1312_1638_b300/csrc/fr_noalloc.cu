// fr_rk4_noalloc: the RK4 step without any device allocation at call time.
//
// fr_rk4 keeps its two RK4 stage registers in device memory that it obtains
// with cudaMalloc on its first call.  Some callers cannot let a library do
// that: host applications whose framework reserves the GPU's memory up front
// and hands it out from its own pool (a cudaMalloc behind its back fails or
// fragments that pool), and time-critical loops that must not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device.
// This entry point gives them the same RK4 step with the registers placed in
// a fixed array compiled into the library (`fr_noalloc_scratch` below), so the
// call itself allocates nothing.  The array lives in this file's own module,
// which the CUDA runtime loads on a device the first time its address is
// looked up there; fr_setup does that look-up on the context's device, so the
// array's FR_NOALLOC_MAX_BYTES are reserved when the context is set up (when
// the library allocates anyway) and stay reserved until the process exits.
#include <cstdio>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/fr.h"
#include "fr_dev.hpp"

namespace {

// The shared scratch: both RK4 registers of every block of one call.
static __device__ __align__(256) unsigned char fr_noalloc_scratch[FR_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch[kMaxDevices] = {};   // device address of fr_noalloc_scratch, per device

// Device address of the array on the current device (set up once per device).
// In host code the symbol's name is only a host-side stand-in; a kernel must
// be given the address that cudaGetSymbolAddress returns for this device.
cudaError_t scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_scratch[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, fr_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[device] = p;
    }
    *out = g_scratch[device];
    return cudaSuccess;
}

// stage combination, k in tmp: first stage acc = u + a_acc k, later stages
// acc += a_acc k; then tmp = u + a_tmp k
template <typename T>
__global__ void stage_kernel(int64_t n, T* __restrict__ acc, T* __restrict__ tmp, const T* __restrict__ u,
                             T a_acc, T a_tmp, int first) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T k = tmp[i], ui = u[i];
    acc[i] = (first ? ui : acc[i]) + a_acc * k;
    tmp[i] = ui + a_tmp * k;
}

template <typename T>
__global__ void final_kernel(int64_t n, const T* __restrict__ acc, const T* __restrict__ k, T* __restrict__ u, T a) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    u[i] = acc[i] + a * k[i];
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

template <typename T>
cudaError_t rk4_static(fr::DevCtx& c, void* const* u, double dt, int nsteps, unsigned char* base,
                       cudaStream_t st) {
    const size_t nb = c.blocks.size();
    void* acc[16];
    void* tmp[16];
    size_t off = 0;
    for (size_t b = 0; b < nb; ++b) {
        const fr::DevBlock& B = c.blocks[b];
        size_t bytes = align256((size_t)B.nupts * B.nvars * B.ld * sizeof(T));
        acc[b] = base + off;
        tmp[b] = base + off + bytes;
        off += 2 * bytes;
    }
    const double a_acc[4] = {dt / 6, dt / 3, dt / 3, dt / 6};
    const double a_tmp[3] = {dt / 2, dt / 2, dt};
    for (int step = 0; step < nsteps; ++step) {
        for (int s = 0; s < 4; ++s) {
            // the first stage reads u directly; later stages read the stage state in tmp
            cudaError_t e = fr::launch_rhs(c, s == 0 ? u : tmp, tmp, st);
            if (e != cudaSuccess) return e;
            for (size_t b = 0; b < nb; ++b) {
                const fr::DevBlock& B = c.blocks[b];
                int64_t n = (int64_t)B.nupts * B.nvars * B.ld;
                unsigned grid = (unsigned)((n + 255) / 256);
                if (s < 3)
                    stage_kernel<T><<<grid, 256, 0, st>>>(n, (T*)acc[b], (T*)tmp[b], (const T*)u[b], T(a_acc[s]),
                                                          T(a_tmp[s]), s == 0);
                else
                    final_kernel<T><<<grid, 256, 0, st>>>(n, (const T*)acc[b], (const T*)tmp[b], (T*)u[b],
                                                          T(a_acc[3]));
            }
        }
    }
    return cudaGetLastError();
}

}  // namespace

namespace fr {
// Called by fr_setup with the context's device current: looks up (and so
// reserves) the array on that device, so that fr_rk4_noalloc's calls find
// its address cached.  A failure here is not an error of the set-up; the
// entry point then tries again and reports it.
void noalloc_prepare(int device) {
    void* p = nullptr;
    (void)scratch_address(device, &p);
    (void)cudaGetLastError();
}
}  // namespace fr

extern "C" fr_status fr_rk4_noalloc(fr_ctx* ctx, void* const* u, double dt, int nsteps, void* stream) {
    fr::DevCtx* c = fr::ctx_dev(ctx);
    if (!c || !u || nsteps < 0) return FR_ERR_ARG;
    if (c->device < 0) {
        fr::ctx_set_error(ctx, "host-only context has no device state");
        return FR_ERR_UNSUPPORTED;
    }
    if (fr::ctx_is_part(ctx)) {
        fr::ctx_set_error(ctx, "partitioned context: use fr_rhs_parts for its right-hand side");
        return FR_ERR_UNSUPPORTED;
    }
    if (c->blocks.size() > 16) {
        fr::ctx_set_error(ctx, "fr_rk4_noalloc supports at most 16 element blocks");
        return FR_ERR_ARG;
    }
    for (size_t b = 0; b < c->blocks.size(); ++b)
        if (!u[b]) return FR_ERR_ARG;
    const size_t rs = c->precision == FR_PREC_FP64 ? sizeof(double) : sizeof(float);
    size_t need = 0;
    for (const auto& B : c->blocks) need += 2 * align256((size_t)B.nupts * B.nvars * B.ld * rs);
    if (need > (size_t)FR_NOALLOC_MAX_BYTES) {
        std::string m = "fr_rk4_noalloc: the RK4 registers of this mesh need " + std::to_string(need) +
                        " bytes; the library's static scratch holds " + std::to_string((size_t)FR_NOALLOC_MAX_BYTES) +
                        " bytes (use fr_rk4)";
        fr::ctx_set_error(ctx, m.c_str());
        return FR_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(c->device);
    void* base = nullptr;
    if (e == cudaSuccess) e = scratch_address(c->device, &base);
    if (e != cudaSuccess) {
        fr::ctx_set_error(ctx, cudaGetErrorString(e));
        return FR_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // kernel timing records CUDA events, which the runtime may allocate: it is
    // suspended for this call (its kernels are not timed)
    const bool prof = c->prof;
    c->prof = false;
    e = c->precision == FR_PREC_FP64 ? rk4_static<double>(*c, u, dt, nsteps, (unsigned char*)base, st)
                                     : rk4_static<float>(*c, u, dt, nsteps, (unsigned char*)base, st);
    c->prof = prof;
    if (e != cudaSuccess) {
        fr::ctx_set_error(ctx, cudaGetErrorString(e));
        return FR_ERR_CUDA;
    }
    return FR_OK;
}
