// CUDA-core transform pass (precisions ETD_PREC_FP32 and ETD_PREC_FP64):
//     out(b, mm, nn) = sum_k A[b][mm][k] P[nn][k]   followed by the fused epilogue.
// Shared-memory tiled product, 64 x 64 outputs per block of 256 threads, each
// thread 4 x 4 outputs. Threads along x own consecutive rows mm, so the
// transposed epilogue stores (consecutive mm are consecutive addresses) coalesce.
#include "etd_internal.cuh"

namespace etd {

namespace {
constexpr int SB_M = 64, SB_N = 64, SB_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const T* __restrict__ A, const T* __restrict__ P, int M, int n,
                                                        const Epi<T> e) {
    __shared__ T As[SB_K][SB_M + 1];
    __shared__ T Bs[SB_K][SB_N + 1];
    const int b = blockIdx.z;
    const int m0 = blockIdx.x * SB_M, n0 = blockIdx.y * SB_N;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const T* Ab = A + (long long)b * e.bs;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;

    for (int k0 = 0; k0 < n; k0 += SB_K) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int el = threadIdx.x + 256 * r;  // 64 rows x 16 k
            const int row = el / SB_K, col = el % SB_K;
            const int k = k0 + col;
            const int mm = m0 + row, nn = n0 + row;
            As[col][row] = (mm < M && k < n) ? Ab[(long long)mm * e.ld + k] : (T)0;
            Bs[col][row] = (nn < n && k < n) ? P[(long long)nn * e.ld + k] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SB_K; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mm = m0 + tx + 16 * i;
        if (mm >= M) continue;
        const int mh = mm / n, ml = mm - mh * n;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + ty + 16 * j;
            if (nn < n) e.apply(b, mh, ml, nn, acc[i][j]);
        }
    }
}
}  // namespace

void launch_gemm_simt_f32(const float* A, const float* P, int M, int n, int nbatch, const Epi<float>& e,
                          cudaStream_t st) {
    dim3 grid((M + SB_M - 1) / SB_M, (n + SB_N - 1) / SB_N, nbatch);
    gemm_simt_kernel<float><<<grid, 256, 0, st>>>(A, P, M, n, e);
}

void launch_gemm_simt_f64(const double* A, const double* P, int M, int n, int nbatch, const Epi<double>& e,
                          cudaStream_t st) {
    dim3 grid((M + SB_M - 1) / SB_M, (n + SB_N - 1) / SB_N, nbatch);
    gemm_simt_kernel<double><<<grid, 256, 0, st>>>(A, P, M, n, e);
}

}  // namespace etd
