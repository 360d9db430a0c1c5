// ocean_components.cu -- standalone kernels over caller-owned device buffers: the
// adaptive-order WENO-Z face reconstruction and the batched Thomas solve, the same
// device functions the step kernels use, exposed for component-level checks.
#include <cstdio>
#include <mutex>
#include <string>

#include "ocean.h"
#include "ocean_internal.cuh"

namespace {

template <typename R>
__global__ void k_weno_faces(const R* __restrict__ q, const R* __restrict__ vel,
                             const unsigned char* __restrict__ inside, int n, R* __restrict__ out,
                             R eps, int linear) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const bool pos = vel[f] >= R(0);
    R s[5];
    unsigned in = 0;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        int c = pos ? f - 3 + m : f + 2 - m;
        c %= n;
        if (c < 0) c += n;
        s[m] = q[c];
        in |= ((inside ? inside[c] != 0 : true) ? 1u : 0u) << m;
    }
    out[f] = weno_adaptive(s, in, eps, linear);
}

template <typename R>
__global__ void k_tridiag(const R* __restrict__ a, const R* __restrict__ b, const R* __restrict__ c,
                          const R* __restrict__ d, R* __restrict__ x, int n, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    // forward elimination writes c' into x's slots' companion (kept in registers via a
    // local array bounded by n <= 256) and d' into x; back substitution in place
    R cp[256];
    R inv = R(1) / b[s];
    cp[0] = c[s] * inv;
    x[s] = d[s] * inv;
    for (int k = 1; k < n; ++k) {
        const long e = (long)k * nsys + s;
        const R ak = a[e];
        inv = R(1) / (b[e] - ak * cp[k - 1]);
        cp[k] = c[e] * inv;
        x[e] = (d[e] - ak * x[e - nsys]) * inv;
    }
    for (int k = n - 2; k >= 0; --k) {
        const long e = (long)k * nsys + s;
        x[e] = x[e] - cp[k] * x[e + nsys];
    }
}

}  // namespace

extern "C" {

int ocean_weno_faces(const void* d_q, const void* d_vel, const unsigned char* d_inside, int n,
                     void* d_out, int precision, double eps, int linear, void* stream) {
    if (!d_q || !d_vel || !d_out || n < 5) return OCEAN_ERR_ARG;
    const int tpb = 256, nb = (n + tpb - 1) / tpb;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == OCEAN_FP64)
        k_weno_faces<double><<<nb, tpb, 0, s>>>((const double*)d_q, (const double*)d_vel, d_inside,
                                                n, (double*)d_out, eps, linear);
    else if (precision == OCEAN_MIXED)
        k_weno_faces<float><<<nb, tpb, 0, s>>>((const float*)d_q, (const float*)d_vel, d_inside, n,
                                               (float*)d_out, (float)eps, linear);
    else
        return OCEAN_ERR_ARG;
    return cudaGetLastError() == cudaSuccess ? OCEAN_OK : OCEAN_ERR_CUDA;
}

int ocean_tridiag_batched(const void* d_a, const void* d_b, const void* d_c, const void* d_d,
                          void* d_x, int n, int nsys, int precision, void* stream) {
    if (!d_a || !d_b || !d_c || !d_d || !d_x || n < 1 || n > 256 || nsys < 1) return OCEAN_ERR_ARG;
    const int tpb = 128, nb = (nsys + tpb - 1) / tpb;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == OCEAN_FP64)
        k_tridiag<double><<<nb, tpb, 0, s>>>((const double*)d_a, (const double*)d_b,
                                             (const double*)d_c, (const double*)d_d, (double*)d_x,
                                             n, nsys);
    else if (precision == OCEAN_MIXED)
        k_tridiag<float><<<nb, tpb, 0, s>>>((const float*)d_a, (const float*)d_b, (const float*)d_c,
                                            (const float*)d_d, (float*)d_x, n, nsys);
    else
        return OCEAN_ERR_ARG;
    return cudaGetLastError() == cudaSuccess ? OCEAN_OK : OCEAN_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Batched tridiagonal solve without any allocation.
//
// For callers that must not allocate device memory: code embedded in another framework
// whose caching allocator owns the device's free memory, a runtime with a fixed memory
// budget, or a latency-bound loop that must not make the device-synchronising
// cudaMalloc/cudaFree calls.  The solve above keeps the Thomas coefficients c' in a per-thread
// local-memory frame that the driver sets aside at launch; this variant keeps them,
// level-major, in one file-scope device array instead, so the call needs no memory
// beyond the caller's inputs and outputs and this module's static storage.
//
// The array holds OCEAN_TRIDIAG_STATIC_WORDS 8-byte words (16 MiB) on every GPU that
// loads the library, until the process exits: n * nsys may not exceed that many
// doubles, or twice that many floats.  Every call uses the same array and leaves its
// coefficients there; nothing needs clearing, because each call writes every element
// it reads before reading it.  Calls whose execution overlaps on the GPU (different
// streams, or different host threads) race on the array and must be serialised.

static __device__ __align__(256) double g_tridiag_cp[OCEAN_TRIDIAG_STATIC_WORDS];

namespace {

// c'(k, s) lives at cp[k * nsys + s]: the threads of a warp touch consecutive words
template <typename R>
__global__ void k_tridiag_static(const R* __restrict__ a, const R* __restrict__ b,
                                 const R* __restrict__ c, const R* __restrict__ d,
                                 R* __restrict__ x, R* __restrict__ cp, int n, int nsys) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    R inv = R(1) / b[s];
    R cprev = c[s] * inv;
    cp[s] = cprev;
    x[s] = d[s] * inv;
    for (int k = 1; k < n; ++k) {
        const long e = (long)k * nsys + s;
        const R ak = a[e];
        inv = R(1) / (b[e] - ak * cprev);
        cprev = c[e] * inv;
        cp[e] = cprev;
        x[e] = (d[e] - ak * x[e - nsys]) * inv;
    }
    for (int k = n - 2; k >= 0; --k) {
        const long e = (long)k * nsys + s;
        x[e] = x[e] - cp[e] * x[e + nsys];
    }
}

// device address of the static array on the current device, looked up once per device
// and kept for the life of the process (a device reset would make it stale)
std::mutex g_static_mu;
void* g_static_ptr[128];

int static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        oc_set_last_error(cudaGetErrorString(e));
        return OCEAN_ERR_CUDA;
    }
    if (dev < 0 || dev >= 128) {
        oc_set_last_error("device index out of range for the static scratch table");
        return OCEAN_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tridiag_cp);
        if (e != cudaSuccess || !p) {
            oc_set_last_error(e != cudaSuccess ? cudaGetErrorString(e)
                                               : "cudaGetSymbolAddress returned null");
            return OCEAN_ERR_CUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return OCEAN_OK;
}

}  // namespace

extern "C" int ocean_tridiag_batched_static(const void* d_a, const void* d_b, const void* d_c,
                                            const void* d_d, void* d_x, int n, int nsys,
                                            int precision, void* stream) {
    if (!d_a || !d_b || !d_c || !d_d || !d_x) {
        oc_set_last_error("ocean_tridiag_batched_static: null array");
        return OCEAN_ERR_ARG;
    }
    if (n < 1 || nsys < 1) {
        oc_set_last_error("ocean_tridiag_batched_static: n and nsys must be >= 1");
        return OCEAN_ERR_ARG;
    }
    if (precision != OCEAN_FP64 && precision != OCEAN_MIXED) {
        oc_set_last_error("ocean_tridiag_batched_static: unknown precision");
        return OCEAN_ERR_ARG;
    }
    const size_t esz = precision == OCEAN_FP64 ? sizeof(double) : sizeof(float);
    const size_t cap = sizeof(g_tridiag_cp) / esz;
    if ((size_t)n * (size_t)nsys > cap) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "ocean_tridiag_batched_static: n * nsys = %zu exceeds the static scratch of %zu "
                 "elements (%zu bytes)", (size_t)n * (size_t)nsys, cap, sizeof(g_tridiag_cp));
        oc_set_last_error(msg);
        return OCEAN_ERR_ARG;
    }
    void* cp = nullptr;
    int rc = static_scratch(&cp);
    if (rc != OCEAN_OK) return rc;
    const int tpb = 128, nb = (nsys + tpb - 1) / tpb;
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == OCEAN_FP64)
        k_tridiag_static<double><<<nb, tpb, 0, s>>>((const double*)d_a, (const double*)d_b,
                                                    (const double*)d_c, (const double*)d_d,
                                                    (double*)d_x, (double*)cp, n, nsys);
    else
        k_tridiag_static<float><<<nb, tpb, 0, s>>>((const float*)d_a, (const float*)d_b,
                                                   (const float*)d_c, (const float*)d_d,
                                                   (float*)d_x, (float*)cp, n, nsys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        oc_set_last_error(cudaGetErrorString(e));
        return OCEAN_ERR_CUDA;
    }
    return OCEAN_OK;
}
