// Fast sine transform pass (ETD_PREC_DST32): the comparison path in which every
// transform pass is a set of DST-I transforms computed with FFTs instead of the
// dense product with P. P is the DST-I matrix, P[j][k] = sqrt(2/(n+1)) sin(pi
// (j+1)(k+1)/(n+1)), so one pass out(b, mm, k) = sum_j A[b][mm][j] P[k][j] is a
// DST-I of every row of A: O(n log n) per row instead of O(n^2).
//
// DST-I through a complex FFT of length N = 2(n+1): the odd extension
//   z_0 = 0, z_j = x_{j-1} (1 <= j <= n), z_{n+1} = 0, z_{N-j} = -z_j
// has the purely imaginary DFT Z_k = -2i sum_j x_j sin(pi j' k/(n+1)) (j' = j+1),
// so y_k = -Im Z_{k+1} / 2. Two real rows a and b ride in one complex FFT
// (z = z_a + i z_b): Z = i A - B with A, B real, so y_a = -Im Z / 2 and
// y_b = Re Z / 2. The FFT is an iterative decimation in time in shared memory,
// three radix-2 stages per round (radix 8) after one single stage or one radix-4
// round when log2 N is not a multiple of 3. Twiddles come from a host table computed in FP64 and laid out by stage
// (stage s, half = 2^s: entries half - 1 + pos = e^{-i pi pos / half}), so the
// lanes of a warp read consecutive entries; read with the stride of one table
// e^{-2 pi i k / N} they all hit one shared-memory bank.
//
// The row kernel writes the transformed rows in natural order to a scratch
// buffer; the transpose kernel reads them through 32 x 32 shared-memory tiles
// and applies the pass's fused epilogue (split, Hadamard stage, physical
// field) at the transposed position, so both kernels access memory coalesced.
#include <cuda_runtime.h>

#include <cmath>

#include "etd_internal.cuh"

namespace etd {

namespace {

// Shared-memory index of element i of a transform: one padding slot after every
// 32 elements, so that the strided accesses of the bit-reversed stores and of
// the butterflies of early stages spread over the banks.
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }

// One radix-2 butterfly with twiddle w: (a, b) <- (a + w b, a - w b).
__device__ __forceinline__ void bfly(float2& a, float2& b, float2 w) {
    const float2 t = make_float2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
    b = make_float2(a.x - t.x, a.y - t.y);
    a = make_float2(a.x + t.x, a.y + t.y);
}

// G row pairs per block iteration (G N = 4096 complex values for short rows), so
// that one barrier per butterfly stage serves several transforms. Row r of the
// stacked components starts at r * ld in both A and out (component stride M ld).
__global__ void __launch_bounds__(512) dst_rows_kernel(const float* __restrict__ A, long long R, int n, int ld,
                                                       const float2* __restrict__ tw, int logN, int logG, float scale,
                                                       float* __restrict__ out) {
    extern __shared__ float2 z[];
    const int N = 1 << logN, G = 1 << logG;
    const int NP = N + (N >> 5);  // padded length of one transform
    const long long pairs = (R + 1) / 2;
    const long long groups = (pairs + G - 1) / G;
    for (long long gr = blockIdx.x; gr < groups; gr += gridDim.x) {
        // odd extensions of both rows of each pair, stored at bit-reversed positions
        for (int g = 0; g < G; ++g) {
            const long long ra = 2 * (gr * G + g), rb = ra + 1;
            const float* xa = A + ra * ld;
            const float* xb = A + rb * ld;
            const bool has_a = ra < R, has_b = rb < R;
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                float re = 0.f, im = 0.f;
                if (j >= 1 && j <= n) {
                    if (has_a) re = xa[j - 1];
                    if (has_b) im = xb[j - 1];
                } else if (j >= n + 2) {
                    if (has_a) re = -xa[N - j - 1];
                    if (has_b) im = -xb[N - j - 1];
                }
                z[g * NP + pad32((int)(__brev((unsigned)j) >> (32 - logN)))] = make_float2(re, im);
            }
        }
        __syncthreads();
        // stages 0 .. logN-1: one radix-2 stage or one radix-4 round first when
        // log2 N is not a multiple of 3, then radix-8 rounds (three stages per
        // shared-memory round trip)
        int s = 0;
        if (logN % 3 == 1) {  // radix-2 stage (half = 1)
            for (int qq = threadIdx.x; qq < ((N / 2) << logG); qq += blockDim.x) {
                const int g = qq >> (logN - 1), q = qq & (N / 2 - 1);
                const int pi = g * NP + pad32(2 * q), pj = g * NP + pad32(2 * q + 1);
                const float2 a = z[pi], b = z[pj];
                z[pi] = make_float2(a.x + b.x, a.y + b.y);
                z[pj] = make_float2(a.x - b.x, a.y - b.y);
            }
            __syncthreads();
            s = 1;
        } else if (logN % 3 == 2) {  // radix-4 round: stages 0 (half = 1) and 1
            for (int qq = threadIdx.x; qq < ((N / 4) << logG); qq += blockDim.x) {
                const int g = qq >> (logN - 2), q = qq & (N / 4 - 1);
                const int i0 = q << 2;
                const int p0 = g * NP + pad32(i0), p1 = g * NP + pad32(i0 + 1);
                const int p2 = g * NP + pad32(i0 + 2), p3 = g * NP + pad32(i0 + 3);
                float2 x0 = z[p0], x1 = z[p1], x2 = z[p2], x3 = z[p3];
                bfly(x0, x1, tw[0]);
                bfly(x2, x3, tw[0]);
                bfly(x0, x2, tw[1]);
                bfly(x1, x3, tw[2]);
                z[p0] = x0;
                z[p1] = x1;
                z[p2] = x2;
                z[p3] = x3;
            }
            __syncthreads();
            s = 2;
        }
        for (; s < logN; s += 3) {  // radix-8 rounds: stages s (half), s + 1, s + 2 in registers
            const int half = 1 << s;
            for (int qq = threadIdx.x; qq < ((N / 8) << logG); qq += blockDim.x) {
                const int g = qq >> (logN - 3), q = qq & (N / 8 - 1);
                const int pos = q & (half - 1);
                const int i0 = ((q >> s) << (s + 3)) + pos;
                int pk[8];
                float2 x[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    pk[k] = g * NP + pad32(i0 + k * half);
                    x[k] = z[pk[k]];
                }
                const float2 w1 = tw[half - 1 + pos];  // stage s
#pragma unroll
                for (int a = 0; a < 8; a += 2) bfly(x[a], x[a + 1], w1);
                const float2 wa = tw[2 * half - 1 + pos], wb = tw[2 * half - 1 + pos + half];  // stage s + 1
                bfly(x[0], x[2], wa);
                bfly(x[1], x[3], wb);
                bfly(x[4], x[6], wa);
                bfly(x[5], x[7], wb);
#pragma unroll
                for (int k = 0; k < 4; ++k) bfly(x[k], x[k + 4], tw[4 * half - 1 + pos + k * half]);  // stage s + 2
#pragma unroll
                for (int k = 0; k < 8; ++k) z[pk[k]] = x[k];
            }
            __syncthreads();
        }
        const float h = 0.5f * scale;
        for (int g = 0; g < G; ++g) {
            const long long ra = 2 * (gr * G + g), rb = ra + 1;
            if (ra >= R) break;
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                const float2 c = z[g * NP + pad32(k + 1)];
                out[ra * ld + k] = -c.y * h;
                if (rb < R) out[rb * ld + k] = c.x * h;
            }
        }
        __syncthreads();  // z is reused by the next group
    }
}

// out(b, mm, nn) from the natural-order rows tmp[b * M + mm][nn] through the
// pass epilogue; a 32 x 32 tile per block, lanes along mm on the write side.
__global__ void __launch_bounds__(256) dst_transpose_epi_kernel(const float* __restrict__ tmp, int M, int n,
                                                                int nbatch, int ld, const Epi<float> e) {
    __shared__ float tile[32][33];
    const long long R = (long long)nbatch * M;
    const long long r0 = (long long)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const long long r = r0 + i;
        const int c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < R && c < n) ? tmp[r * ld + c] : 0.f;
    }
    __syncthreads();
    const long long r = r0 + threadIdx.x;
    if (r >= R) return;
    const int b = (int)(r / M), mm = (int)(r - (long long)b * M);
    const int mh = mm / n, ml = mm - mh * n;
    // four consecutive columns per thread (blockDim.y = 8): their state loads go
    // out together, then the batched epilogue
    const int i0 = 4 * threadIdx.y, nn0 = c0 + i0;
    if (nn0 >= n) return;
    const int count = min(4, n - nn0);
    float2 st[4];
    epi_load_state<4>(e, b, mh, ml, nn0, count, st);
    float v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = tile[threadIdx.x][i0 + i];
    epi_apply_batch<4>(e, b, mh, ml, nn0, v, count, st);
}

}  // namespace

cudaError_t launch_dst_pass(const float* A, int M, int n, int nbatch, int ld, long long bs, const float2* tw,
                            float* tmp, const Epi<float>& e, cudaStream_t st) {
    int logN = 0;
    while ((1 << logN) < 2 * (n + 1)) ++logN;
    if ((1 << logN) != 2 * (n + 1) || logN < 5 || logN > 14) return cudaErrorInvalidValue;
    if (bs != (long long)M * ld) return cudaErrorInvalidValue;  // rows of all components at r * ld
    const int logG = logN < 12 ? 12 - logN : 0;  // row pairs per block iteration
    const int np = (1 << logN) + (1 << logN) / 32;
    const size_t smem = sizeof(float2) * ((size_t)np << logG);
    static bool attr = false;
    if (!attr) {
        cudaError_t ce = cudaFuncSetAttribute(dst_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(sizeof(float2) * ((1 << 14) + (1 << 9))));
        if (ce != cudaSuccess) return ce;
        attr = true;
    }
    const long long R = (long long)nbatch * M;
    const long long groups = ((R + 1) / 2 + (1 << logG) - 1) >> logG;
    const unsigned grid = (unsigned)(groups < 152LL * 16 ? groups : 152LL * 16);
    const float scale = (float)std::sqrt(2.0 / (double)(n + 1));
    dst_rows_kernel<<<grid, 512, smem, st>>>(A, R, n, ld, tw, logN, logG, scale, tmp);
    const dim3 tg((unsigned)((R + 31) / 32), (unsigned)((n + 31) / 32));
    dst_transpose_epi_kernel<<<tg, dim3(32, 8), 0, st>>>(tmp, M, n, nbatch, ld, e);
    return cudaGetLastError();
}

}  // namespace etd
