// etd_transform_noalloc: the spectral transform of a field without any device
// allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// transform: code that runs inside a host framework whose caching allocator
// has reserved the GPU's memory up front (a cudaMalloc outside that pool can
// fail or fragment it), and latency-critical loops where cudaFree, which
// synchronises the whole device, would stall every other stream. For them this
// entry point takes only the input and output fields and keeps its workspace
// (the sine basis P and the intermediate passes) in a statically sized device
// array that is part of the library image.
//
// The workspace is g_noalloc_scratch below: ETD_NOALLOC_MAX_ELEMS floats
// (16 MiB). Every GPU that loads the library holds it until the process exits.
// In host code the name of a __device__ array is only a host-side stand-in, so
// the entry point looks up its device address once per device and CUDA context
// with cudaGetSymbolAddress (with that device current) and passes that pointer
// to the kernels. The context's unique id (cuCtxGetId) is kept with the address:
// after cudaDeviceReset the runtime creates a new context, the module and its
// array are loaded again at a new address, and the next call repeats the set-up.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/etd.h"
#include "etd_internal.cuh"

namespace {

__device__ __align__(256) float g_noalloc_scratch[ETD_NOALLOC_MAX_ELEMS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
float* g_scratch_ptr[MAX_DEVICES] = {nullptr};
unsigned long long g_scratch_ctx[MAX_DEVICES] = {0};  // context id the address belongs to (0: unknown)

// Unique id of the current context through the driver entry points (no link
// against libcuda); 0 when the driver does not offer them.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// P[j][k] = sqrt(2/(n+1)) sin(pi (j+1)(k+1)/(n+1)), the orthonormal sine
// eigenvectors of the 1D Dirichlet second difference (Section 3.3.2's P_x).
__global__ void noalloc_build_p(float* __restrict__ P, int n) {
    const long long total = (long long)n * n;
    const double scale = sqrt(2.0 / (n + 1));
    const long long period = 2LL * (n + 1);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long j = i / n, k = i - j * n;
        const long long r = ((j + 1) * (k + 1)) % period;
        P[i] = (float)(scale * sinpi((double)r / (double)(n + 1)));
    }
}

// One transform pass with FP32 CUDA-core products, unpadded rows:
//   out(b, mm, nn) = sum_k A[b][mm][k] P[nn][k],
// stored at ((nn * mq + mm / n) * n + mm % n) of component b, so that the
// contracted axis becomes the slowest one (2 passes = P X P, 3 = mode products).
constexpr int TB = 64, TK = 16;
__global__ void __launch_bounds__(256) noalloc_pass(const float* __restrict__ A, const float* __restrict__ P,
                                                    float* __restrict__ out, int M, int n, int mq) {
    __shared__ float As[TK][TB + 1];
    __shared__ float Bs[TK][TB + 1];
    const int b = blockIdx.z;
    const int m0 = blockIdx.x * TB, n0 = blockIdx.y * TB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const long long cs = (long long)M * n;  // component stride
    const float* Ab = A + b * cs;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < n; k0 += TK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int el = threadIdx.x + 256 * r;
            const int row = el / TK, col = el % TK, k = k0 + col;
            As[col][row] = (m0 + row < M && k < n) ? Ab[(long long)(m0 + row) * n + k] : 0.f;
            Bs[col][row] = (n0 + row < n && k < n) ? P[(long long)(n0 + row) * n + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* ob = out + b * cs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mm = m0 + tx + 16 * i;
        if (mm >= M) continue;
        const int mh = mm / n, ml = mm - mh * n;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + ty + 16 * j;
            if (nn < n) ob[((long long)nn * mq + mh) * n + ml] = acc[i][j];
        }
    }
}

etd_status fail_noalloc(etd_status s, const char* msg) {
    etd::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" etd_status etd_transform_noalloc(int d, int n, int n_comp, const void* in_dev, void* out_dev,
                                            void* stream) {
    if (d != 2 && d != 3) return fail_noalloc(ETD_ERR_INVALID_ARG, "etd_transform_noalloc: d must be 2 or 3");
    if (n < 2) return fail_noalloc(ETD_ERR_INVALID_ARG, "etd_transform_noalloc: n must be >= 2");
    if (n_comp < 1 || n_comp > 2) return fail_noalloc(ETD_ERR_INVALID_ARG, "etd_transform_noalloc: n_comp must be 1 or 2");
    if (!in_dev || !out_dev) return fail_noalloc(ETD_ERR_INVALID_ARG, "etd_transform_noalloc: NULL field pointer");
    const long long npts = (d == 2) ? (long long)n * n : (long long)n * n * n;
    const long long field = (long long)n_comp * npts;
    const long long need = (long long)n * n + (d == 3 ? 2 : 1) * field;
    if (need > (long long)ETD_NOALLOC_MAX_ELEMS) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "etd_transform_noalloc: d=%d n=%d n_comp=%d needs %lld workspace floats, more than the static "
                 "maximum ETD_NOALLOC_MAX_ELEMS = %d",
                 d, n, n_comp, need, ETD_NOALLOC_MAX_ELEMS);
        return fail_noalloc(ETD_ERR_INVALID_ARG, msg);
    }
    int dev = -1;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return fail_noalloc(ETD_ERR_CUDA, "etd_transform_noalloc: no current CUDA device");
    float* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_ptr[dev] || ctx != g_scratch_ctx[dev]) {
            // set-up, once per device and context: device address of the static workspace
            void* ptr = nullptr;
            ce = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (ce != cudaSuccess) {
                char msg[256];
                snprintf(msg, sizeof msg, "etd_transform_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(ce));
                return fail_noalloc(ETD_ERR_CUDA, msg);
            }
            g_scratch_ptr[dev] = static_cast<float*>(ptr);
            // the lookup made the device's context current if none was: record that one
            g_scratch_ctx[dev] = current_context_id();
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    float* P = base;
    float* buf0 = base + (long long)n * n;
    float* buf1 = buf0 + field;
    const int M = (d == 2) ? n : n * n;
    const int mq = (d == 2) ? 1 : n;
    // every workspace value read below is written earlier in this call, so
    // nothing has to be cleared
    long long pblocks = ((long long)n * n + 255) / 256;
    if (pblocks > 4096) pblocks = 4096;
    // Each launch is checked through its own return code (cudaLaunchKernel), so
    // an error some earlier work of the caller left pending is neither reported
    // as this call's failure nor cleared.
    int nn = n;
    void* pargs[] = {&P, &nn};
    ce = cudaLaunchKernel((const void*)noalloc_build_p, dim3((unsigned)pblocks), dim3(256), pargs, 0, st);
    const dim3 grid((M + TB - 1) / TB, (n + TB - 1) / TB, n_comp);
    const float* chain[4] = {static_cast<const float*>(in_dev), buf0, d == 2 ? static_cast<float*>(out_dev) : buf1,
                             static_cast<float*>(out_dev)};
    int MM = M, mqq = mq;
    for (int pass = 0; pass < d && ce == cudaSuccess; ++pass) {
        const float* a = chain[pass];
        float* o = const_cast<float*>(chain[pass + 1]);
        void* args[] = {&a, &P, &o, &MM, &nn, &mqq};
        ce = cudaLaunchKernel((const void*)noalloc_pass, grid, dim3(256), args, 0, st);
    }
    if (ce != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "etd_transform_noalloc: launch failed: %s", cudaGetErrorString(ce));
        return fail_noalloc(ETD_ERR_CUDA, msg);
    }
    return ETD_OK;
}
