// Tensor-core transform pass for sm_103a (precisions ETD_PREC_TF32, ETD_PREC_TF32X3):
//     out(b, mm, nn) = sum_k A[b][mm][k] P[nn][k]     + fused epilogue (etd_internal.cuh)
//
// Split TF32 (Section 3.3.2's products done on 5th-generation tensor cores):
// every operand is stored as hi = rna_tf32(x), lo = rna_tf32(x - hi), and one
// tile accumulates hi*hi + hi*lo + lo*hi in FP32 in tensor memory, which keeps
// about 21 bits of each product instead of TF32's 11.
//
// One CTA computes a 128 x bn tile (bn <= 256) with 6 warps:
//   warps 0-3  epilogue: tcgen05.ld of the accumulator lanes 32w..32w+31, the
//              Hadamard stage of eq. (13)/(14) when this pass ends a transform,
//              transposed (coalesced) stores;
//   warp 4     TMA producer (one lane) and tensor-memory allocator (whole warp);
//   warp 5     MMA issuer (one lane): tcgen05.mma.cta_group::1.kind::tf32.
// Shared memory holds `stages` k-blocks of 32 FP32 values (128-byte rows,
// 128-byte swizzle, the canonical K-major layout of the MMA descriptors) for
// A hi/lo and P hi/lo. Producer and MMA meet on full/empty mbarriers; the
// accumulator is handed to the epilogue through one more mbarrier signalled by
// tcgen05.commit.
//
// Every wait has a time limit (%globaltimer, 2 s). When one expires the CTA
// raises ERR_TIMEOUT in the plan's error word, stops issuing work, waits (with
// a limit) for its own copies and products in flight, frees its tensor memory
// and returns; later CTAs of the grid see the error word and return at once.
#include <cuda.h>
#include <stdio.h>

#include "etd_internal.cuh"
#include "tc_ptx.cuh"

namespace etd {

struct TcMaps {
    CUtensorMap a[4][3];  // operand buffer i, piece j (hi, mid, lo)
    CUtensorMap p[2][3];  // P pieces, boxes as tall as the tile width of config slot 0 / 1
    int n_a;
};

namespace {

constexpr int BM = 128;
constexpr int BKF = 32;                  // TF32 values per k-block (64 for BF16): 128 bytes of K, the
                                         // span one TMEM accumulator buffer takes before it is drained
constexpr int ROW = 128;                 // bytes of K per operand row in one pipeline stage (64 measured slower)
constexpr int SPD = 128 / ROW;           // pipeline stages per k-block
constexpr int KK = ROW / 32;             // MMAs per stage (each takes 32 bytes of K)
constexpr int A_BYTES = BM * ROW;        // one operand piece of a stage
constexpr int NUM_EPI_WARPS = 8;         // two per TMEM lane quarter, one per column half
constexpr int WARP_TMA = 8;
constexpr int WARP_MMA = 9;
constexpr int WARP_MMA2 = 10;             // ACCURATE: issues the correction products
constexpr int NUM_THREADS = 352;
constexpr int MAX_HALF = 128;            // columns per epilogue warp (bn <= 256)
constexpr int EPI_CS = 36;               // staged column stride (floats): 32 rows + 4, no bank conflicts
constexpr int STAGE_BYTES_EPI = NUM_EPI_WARPS * EPI_CS * MAX_HALF * 4;
constexpr int SMEM_LIMIT = 227 * 1024 - 1024;  // dynamic bytes; leaves room for the static barriers

struct KParams {
    int M, n, bn, stages, products, pieces, tiles_m, tiles_n, tmem_cols;
    int acc_cols;  // columns of one accumulator region (power of two >= bn)
    int nbatch;
    int vec;  // row-vector epilogue (epi_rows8_ok)
    unsigned stage_bytes, b_bytes, tx_bytes;
    unsigned* err;
    Epi<float> e;
};

// Shared-memory matrix descriptor of the pipeline stages (rows of ROW bytes),
// matching the tensor maps' swizzle.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) { return sdesc_kmajor(addr, ROW); }

// sum += v (ACCURATE: compensated, Knuth's 2Sum keeps the rounding error in comp)
template <bool ACCURATE>
__device__ __forceinline__ void acc_add(float& sum, float& comp, float v) {
    if constexpr (ACCURATE) {
        const float t = sum + v;
        const float z = t - sum;
        comp += (sum - (t - z)) + (v - z);
        sum = t;
    } else {
        sum += v;
    }
}

// ACCURATE = false: every product of a k-step into the k-block accumulator,
//   FP32 round-to-nearest running sums (the per-step passes).
// ACCURATE = true (bn <= 128, three operand pieces): only hi*hi goes to the
//   k-block accumulator; the five correction products accumulate over the whole
//   K range in a third TMEM region, and the k-block sums are added with
//   compensated (2Sum) FP32 arithmetic. Used for the transforms whose error
//   stays in the result: U -> U^ when the carried state is (re)built and the
//   transform that returns the field.
template <bool ACCURATE, bool BF16>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    gemm_tf32_tc_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                        const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mP0,
                        const __grid_constant__ CUtensorMap mP1, const __grid_constant__ CUtensorMap mP2,
                        const KParams p) {
    constexpr int KV = BF16 ? 2 * BKF : BKF;  // operand values per k-block
    constexpr int KVS = KV / SPD;             // operand values per pipeline stage
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_skip;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_consumed;
    __shared__ int s_issued;
    // full[8], empty[8] (shared-memory ring), acc_full[2], acc_empty[2] (TMEM ring), done
    __shared__ __align__(8) uint64_t s_bar[8 + 8 + 2 + 2 + 1];

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) s_skip = (*(volatile unsigned*)p.err != 0u);
    __syncthreads();
    if (s_skip) return;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int S = p.stages;
    volatile int* abort_flag = &s_abort;
    const uint32_t bar_full = smem_u32(&s_bar[0]);
    const uint32_t bar_empty = smem_u32(&s_bar[8]);
    const uint32_t bar_acc_full = smem_u32(&s_bar[16]);
    const uint32_t bar_acc_empty = smem_u32(&s_bar[18]);
    const uint32_t bar_done = smem_u32(&s_bar[20]);

    int tm, tn;
    tile_coords(blockIdx.x, p.tiles_m, p.tiles_n, 16, tm, tn);
    const int nst = (p.n + KVS - 1) / KVS;  // pipeline stages of the K range
    const int nk = (nst + SPD - 1) / SPD;   // k-blocks (accumulator buffers drained)
    // TMEM columns: [0, acc) and [acc, 2 acc) k-block buffers, [2 acc, 3 acc) corrections (ACCURATE)
    const uint32_t acc_cols = (uint32_t)p.acc_cols;

    // ACCURATE: two issuing threads (hi*hi, corrections) commit to each stage's
    // `empty` barrier and to `done`
    constexpr uint32_t ISSUERS = ACCURATE ? 2 : 1;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, ISSUERS);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(bar_acc_full + 8 * a, 1);
            mbar_init(bar_acc_empty + 8 * a, NUM_EPI_WARPS);
        }
        mbar_init(bar_done, ISSUERS);
        s_abort = 0;
        s_consumed = 0;
        s_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == WARP_TMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == WARP_TMA && lane == 0) {
        // ---------------- TMA producer ----------------
        const int arow = tm * BM;
        const int prow = tn * p.bn;
        int issued = 0;
        for (int q = 0; q < nst; ++q) {
            const int s = q % S;
            const uint32_t ph = (uint32_t)((q / S) & 1);
            if (!mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort_flag, p.err)) break;
            const uint32_t st = smem_u32(smem + (size_t)s * p.stage_bytes);
            const uint32_t fb = bar_full + 8 * s;
            mbar_expect_tx(fb, p.tx_bytes);
            const int k0 = q * KVS;
            const uint32_t sb = st + (uint32_t)p.pieces * A_BYTES;  // first P piece
            tma_load_2d(st, &mA0, fb, k0, arow);
            tma_load_2d(sb, &mP0, fb, k0, prow);
            if (p.pieces > 1) {
                tma_load_2d(st + A_BYTES, &mA1, fb, k0, arow);
                tma_load_2d(sb + p.b_bytes, &mP1, fb, k0, prow);
            }
            if (p.pieces > 2) {
                tma_load_2d(st + 2 * A_BYTES, &mA2, fb, k0, arow);
                tma_load_2d(sb + 2 * p.b_bytes, &mP2, fb, k0, prow);
            }
            issued = q + 1;
        }
        s_issued = issued;
    } else if (warp == WARP_MMA && lane == 0) {
        // ---------------- MMA issuer: one k-block per accumulator buffer ----------------
        const uint32_t idesc = BF16 ? idesc_bf16(BM, p.bn) : idesc_tf32(BM, p.bn);
        const uint64_t desc0 = sdesc_sw128(smem_u32(smem));  // stage 0, piece 0
        for (int q = 0; q < nst; ++q) {
            const int s = q % S;
            const int kb = q / SPD, a = kb & 1;
            const bool first = q % SPD == 0, last = q % SPD == SPD - 1 || q == nst - 1;  // of the k-block
            if (!mbar_wait(bar_full + 8 * s, (uint32_t)((q / S) & 1), abort_flag, p.err)) break;
            if (first && kb >= 2 &&
                !mbar_wait(bar_acc_empty + 8 * a, (uint32_t)(((kb >> 1) - 1) & 1), abort_flag, p.err))
                break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)a * acc_cols;
            const uint32_t dc = ACCURATE ? tmem + 2u * acc_cols : d;  // correction products
            // operand descriptors by offset from the stage's first one (the start
            // address field is address / 16): the issuing thread keeps up with
            // 128 x 128 x 16 BF16 products only without rebuilding descriptors
            const uint64_t dA0 = desc0 + (uint64_t)(s * (p.stage_bytes >> 4));
            const uint64_t dA1 = dA0 + (A_BYTES >> 4), dA2 = dA0 + 2 * (A_BYTES >> 4);
            const uint64_t dB0 = dA0 + (uint64_t)(p.pieces * (A_BYTES >> 4));
            const uint64_t dB1 = dB0 + (p.b_bytes >> 4), dB2 = dB0 + 2 * (p.b_bytes >> 4);
#pragma unroll
            for (int kk = 0; kk < KK; ++kk) {
                const uint64_t o = 2 * kk;  // 8 TF32 or 16 BF16 values = 32 bytes per MMA
                // terms of (a0 + a1 + a2)(b0 + b1 + b2) down to the 2^-22 level; in
                // ACCURATE mode warp WARP_MMA2 issues the corrections (below)
                mma_op<BF16>(d, dA0 + o, dB0 + o, idesc, (first && kk == 0) ? 0u : 1u);
                if (!ACCURATE && p.products >= 3) {
                    mma_op<BF16>(dc, dA1 + o, dB0 + o, idesc, 1u);
                    mma_op<BF16>(dc, dA0 + o, dB1 + o, idesc, 1u);
                }
                if (!ACCURATE && p.products == 6) {
                    mma_op<BF16>(dc, dA1 + o, dB1 + o, idesc, 1u);
                    mma_op<BF16>(dc, dA2 + o, dB0 + o, idesc, 1u);
                    mma_op<BF16>(dc, dA0 + o, dB2 + o, idesc, 1u);
                }
            }
            mma_commit(bar_empty + 8 * s);                 // stage s may be refilled once these products finish
            if (last) mma_commit(bar_acc_full + 8 * a);  // the k-block sum is ready for the epilogue
            s_consumed = q + 1;
        }
        mma_commit(bar_done);  // arrives when every product issued above has completed
    } else if (ACCURATE && warp == WARP_MMA2 && lane == 0) {
        // ---------------- correction products into their own accumulator ----------------
        // A second issuing thread: the products of a k-block are 4 hi*hi and 20
        // corrections of 128 x bn x 16, and one thread cannot issue them as fast
        // as the tensor core runs them (measured: 2D n = 4096 split BF16 x6, 10.0
        // -> 9.7 ms per step; a third thread with its own region gained nothing).
        // Each thread's commit covers its own products.
        const uint32_t idesc = BF16 ? idesc_bf16(BM, p.bn) : idesc_tf32(BM, p.bn);
        const uint64_t desc0 = sdesc_sw128(smem_u32(smem));
        const uint32_t dc = tmem + 2u * acc_cols;
        for (int q = 0; q < nst; ++q) {
            const int s = q % S;
            if (!mbar_wait(bar_full + 8 * s, (uint32_t)((q / S) & 1), abort_flag, p.err)) break;
            tc_fence_after();
            const uint64_t dA0 = desc0 + (uint64_t)(s * (p.stage_bytes >> 4));
            const uint64_t dA1 = dA0 + (A_BYTES >> 4), dA2 = dA0 + 2 * (A_BYTES >> 4);
            const uint64_t dB0 = dA0 + (uint64_t)(p.pieces * (A_BYTES >> 4));
            const uint64_t dB1 = dB0 + (p.b_bytes >> 4), dB2 = dB0 + 2 * (p.b_bytes >> 4);
#pragma unroll
            for (int kk = 0; kk < KK; ++kk) {
                const uint64_t o = 2 * kk;
                if (p.products >= 3) {  // the first product overwrites the region
                    mma_op<BF16>(dc, dA1 + o, dB0 + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                    mma_op<BF16>(dc, dA0 + o, dB1 + o, idesc, 1u);
                }
                if (p.products == 6) {
                    mma_op<BF16>(dc, dA1 + o, dB1 + o, idesc, 1u);
                    mma_op<BF16>(dc, dA2 + o, dB0 + o, idesc, 1u);
                    mma_op<BF16>(dc, dA0 + o, dB2 + o, idesc, 1u);
                }
            }
            mma_commit(bar_empty + 8 * s);
        }
        mma_commit(bar_done);
    } else if (warp < NUM_EPI_WARPS) {
        // ---------------- epilogue: FP32 round-to-nearest sum of the k-block sums ----------------
        const int quarter = warp & 3;         // TMEM lanes 32*quarter .. +31
        const int half = warp >> 2;           // which half of the tile's columns
        const int hcols = p.bn / 2;           // multiple of 16
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * hcols);
        constexpr int HALF = ACCURATE ? MAX_HALF / 2 : MAX_HALF;
        float sum[HALF];
        float comp[ACCURATE ? HALF : 1];  // 2Sum error terms (ACCURATE)
#pragma unroll
        for (int i = 0; i < HALF; ++i) sum[i] = 0.f;
#pragma unroll
        for (int i = 0; i < (ACCURATE ? HALF : 1); ++i) comp[i] = 0.f;
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
            const int a = kb & 1;
            if (!mbar_wait(bar_acc_full + 8 * a, (uint32_t)((kb >> 1) & 1), abort_flag, p.err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t src = lane_base + (uint32_t)a * acc_cols;
            // 32-column loads where the half-width allows, 16-column loads for a tail
#pragma unroll
            for (int g = 0; g < HALF / 32; ++g) {
                if ((g + 1) * 32 <= hcols) {
                    uint32_t r[32];
                    tmem_ld32(src + (uint32_t)(g * 32), r);
                    tmem_wait32(r);
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        acc_add<ACCURATE>(sum[g * 32 + j], comp[ACCURATE ? g * 32 + j : 0], __uint_as_float(r[j]));
                } else if (g * 32 + 16 <= hcols) {
                    uint32_t r[16];
                    tmem_ld16(src + (uint32_t)(g * 32), r);
                    tmem_wait16(r);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        acc_add<ACCURATE>(sum[g * 32 + j], comp[ACCURATE ? g * 32 + j : 0], __uint_as_float(r[j]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_acc_empty + 8 * a) : "memory");
        }
        if constexpr (ACCURATE) {
            // the correction accumulator is complete once every product has finished
            if (ok && !mbar_wait(bar_done, 0u, abort_flag, p.err)) ok = false;
            tc_fence_after();
            if (ok) {
#pragma unroll
                for (int c = 0; c < HALF / 16; ++c) {
                    if (c * 16 < hcols) {
                        uint32_t r[16];
                        tmem_ld16(lane_base + 2u * acc_cols + (uint32_t)(c * 16), r);
                        tmem_wait16(r);
#pragma unroll
                        for (int j = 0; j < 16; ++j) comp[c * 16 + j] += __uint_as_float(r[j]);
                    }
                }
#pragma unroll
                for (int i = 0; i < HALF; ++i) sum[i] += comp[i];
            }
        }
        if (ok && !*abort_flag) {
            // Every product has completed (the last k-block sum was waited for), so
            // the pipeline's shared memory is free: stage this warp's 32 x hcols sums
            // there column-major and apply the epilogue in a rolled loop (one copy
            // of its code instead of one per column).
            float* stage = reinterpret_cast<float*>(smem) + (size_t)warp * EPI_CS * MAX_HALF;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the TMA writes there
#pragma unroll
            for (int c = 0; c < HALF; ++c)
                if (c < hcols) stage[c * EPI_CS + lane] = sum[c];
            __syncwarp();
            const int grow = tm * BM + quarter * 32 + lane;  // row of the stacked components
            if (p.vec) {
                // lane -> column cc of each group of 8, rows rr0 .. rr0+7 (16-byte accesses)
                const int cc = lane >> 2, rr0 = (lane & 3) * 8;
                const int grow0 = tm * BM + quarter * 32 + rr0;
                const int nn0 = tn * p.bn + half * hcols;
                const int cols = min(hcols, p.n - nn0);  // a multiple of 8
                if (grow0 < p.nbatch * p.M) {
                    const int b = grow0 / p.M, mm = grow0 - b * p.M;
                    const int mh = mm / p.n, ml0 = mm - mh * p.n;
                    float4 cur[4], nxt[4];
                    if (cc < cols) epi_load_rows8(p.e, b, mh, ml0, nn0 + cc, cur);
                    for (int c0 = 0; c0 < cols; c0 += 8) {
                        const int c = c0 + cc;
                        if (c + 8 < cols) epi_load_rows8(p.e, b, mh, ml0, nn0 + c + 8, nxt);
                        if (c < cols) {
                            const float4 a0 = *reinterpret_cast<const float4*>(stage + c * EPI_CS + rr0);
                            const float4 a1 = *reinterpret_cast<const float4*>(stage + c * EPI_CS + rr0 + 4);
                            const float v[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                            epi_apply_rows8(p.e, b, mh, ml0, nn0 + c, v, cur);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) cur[i] = nxt[i];
                    }
                }
            } else if (grow < p.nbatch * p.M) {
                const int b = grow / p.M, mm = grow - b * p.M;
                const int mh = mm / p.n, ml = mm - mh * p.n;
                const int nn0 = tn * p.bn + half * hcols;
                const int cols = min(hcols, p.n - nn0);
                // state loads of the next 16 columns go out before this batch's stores
                float2 cur[16], nxt[16];
                epi_load_state<16>(p.e, b, mh, ml, nn0, min(16, cols), cur);
                for (int c0 = 0; c0 < cols; c0 += 16) {
                    if (c0 + 16 < cols) epi_load_state<16>(p.e, b, mh, ml, nn0 + c0 + 16, min(16, cols - c0 - 16), nxt);
                    float v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = stage[(c0 + i < hcols ? c0 + i : 0) * EPI_CS + lane];
                    epi_apply_batch<16>(p.e, b, mh, ml, nn0 + c0, v, min(16, cols - c0), cur);
#pragma unroll
                    for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == WARP_TMA && lane == 0) {
        if (*abort_flag) {
            // copies still in flight after an abort: wait for them (bounded) before exit
            for (int kb = s_consumed; kb < s_issued; ++kb) {
                const int s = kb % S;
                const unsigned long long t0 = globaltimer();
                while (!mbar_try(bar_full + 8 * s, (uint32_t)((kb / S) & 1)) && globaltimer() - t0 < 100000000ull) {
                }
            }
        }
        const unsigned long long t0 = globaltimer();  // every product has completed
        while (!mbar_try(bar_done, 0u) && globaltimer() - t0 < 200000000ull) {
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == WARP_TMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)p.tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Persistent variant of the per-step pass (two operand pieces or one, no
// ACCURATE mode): one CTA per SM walks the tiles blockIdx.x, + gridDim.x, ...
// The tile's epilogue runs while the next tile's products are already issued:
//   warp 12     TMA producer (one lane), TMEM allocator (whole warp)
//   warp 13     MMA issuer (one lane), k-blocks into TMEM buffers 0/1
//   warps 0-7   drain each k-block buffer into FP32 register sums (two warps
//               per TMEM lane quarter, one per 64-column half); at tile end
//               they write the sums into TMEM staging buffer 0/1 (tcgen05.st)
//   warps 8-11  read a staging buffer (tcgen05.ld) and run the epilogue
// TMEM: four 128-column regions, nkb = 2 k-block buffers followed by nsb = 2
// staging buffers (the layout code also handles 3 + 1).
// Shared memory holds only the TMA ring (three 64 KB stages at bn = 128).
namespace pk {
constexpr int BN = 128;
constexpr int HALF = BN / 2;
constexpr int NUM_DRAIN = 8;
constexpr int NUM_STORE = 8;            // two per TMEM lane quarter, one per column half
constexpr int WARP_TMA = 16;
constexpr int WARP_MMA = 17;
constexpr int WARP_MMA2 = 18;           // ACC: issues the correction products
constexpr int THREADS = 19 * 32;
constexpr int EPI_COLS = 8;             // columns per epilogue batch of a store thread
constexpr int EPI_CS = 36;              // transposition buffer column stride (floats)
constexpr int STATIC_SMEM = NUM_STORE * EPI_COLS * EPI_CS * 4 + 1024;  // buffers + barriers and flags
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t KB_COLS = 128;        // one TMEM region (k-block or staging buffer)
}  // namespace pk


// ACC (short K only, no compensated sums): hi*hi into the k-block buffers, the
// correction products into a fourth TMEM region that spans the tile's whole K
// range; the drain warps add it to their sums once the tile's last k-block is
// in, then free it for the next tile (one staging buffer instead of two).
template <bool BF16, bool ACC, bool VEC>
__global__ void __launch_bounds__(pk::THREADS, 1)
    gemm_tf32_persistent_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                                const __grid_constant__ CUtensorMap mA2, const __grid_constant__ CUtensorMap mP0,
                                const __grid_constant__ CUtensorMap mP1, const __grid_constant__ CUtensorMap mP2,
                                const KParams p) {
    constexpr int KV = BF16 ? 2 * BKF : BKF;  // operand values per k-block
    constexpr int KVS = KV / SPD;             // operand values per pipeline stage
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_skip;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_consumed;
    __shared__ int s_issued;
    // full[8], empty[8], kb_full[3], kb_empty[3], stage_full[2], stage_empty[2], done, corr_empty, corr_full
    __shared__ __align__(8) uint64_t s_bar[8 + 8 + 3 + 3 + 2 + 2 + 1 + 1 + 1];
    // VEC: one EPI_COLS x 32-row transposition buffer per store warp (row-vector
    // epilogue; a separate instantiation, as one kernel with both epilogues spills)
    __shared__ __align__(16) float s_epi[VEC ? pk::NUM_STORE * pk::EPI_COLS * pk::EPI_CS : 4];

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) s_skip = (*(volatile unsigned*)p.err != 0u);
    __syncthreads();
    if (s_skip) return;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int S = p.stages;
    volatile int* abort_flag = &s_abort;
    const uint32_t bar_full = smem_u32(&s_bar[0]);
    const uint32_t bar_empty = smem_u32(&s_bar[8]);
    const uint32_t bar_kb_full = smem_u32(&s_bar[16]);
    const uint32_t bar_kb_empty = smem_u32(&s_bar[19]);
    const uint32_t bar_st_full = smem_u32(&s_bar[22]);
    const uint32_t bar_st_empty = smem_u32(&s_bar[24]);
    const uint32_t bar_done = smem_u32(&s_bar[26]);
    const uint32_t bar_corr_empty = smem_u32(&s_bar[27]);
    const uint32_t bar_corr_full = smem_u32(&s_bar[28]);  // ACC: a tile's corrections are complete
    constexpr uint32_t ISSUERS = ACC ? 2 : 1;              // ACC: a second thread issues the corrections
    const int nst = (p.n + KVS - 1) / KVS;  // pipeline stages of a tile's K range
    const int nk = (nst + SPD - 1) / SPD;   // k-blocks of a tile (accumulator buffers drained)
    const int nkb = 2;                 // k-block buffers (3 + 1 measured slower than 2 + 2)
    const int nsb = ACC ? 1 : 2;       // staging buffers
    const uint32_t corr0 = (uint32_t)nkb * pk::KB_COLS;  // ACC: correction accumulator
    const uint32_t staging0 = (uint32_t)(nkb + (ACC ? 1 : 0)) * pk::KB_COLS;
    const int ntiles = p.tiles_m * p.tiles_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, ISSUERS);
        }
        for (int a = 0; a < 3; ++a) {
            mbar_init(bar_kb_full + 8 * a, 1);
            mbar_init(bar_kb_empty + 8 * a, pk::NUM_DRAIN);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(bar_st_full + 8 * a, pk::NUM_DRAIN);
            mbar_init(bar_st_empty + 8 * a, pk::NUM_STORE);
        }
        mbar_init(bar_done, ISSUERS);
        mbar_init(bar_corr_empty, pk::NUM_DRAIN);
        mbar_init(bar_corr_full, 1);
        s_abort = 0;
        s_consumed = 0;
        s_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == pk::WARP_TMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(pk::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == pk::WARP_TMA && lane == 0) {
        // ---------------- TMA producer: one ring across all tiles ----------------
        int g = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, p.tiles_m, p.tiles_n, 12, tm, tn);
            const int arow = tm * BM;
            const int prow = tn * p.bn;
            for (int q = 0; q < nst; ++q, ++g) {
                const int s = g % S;
                if (!mbar_wait(bar_empty + 8 * s, (uint32_t)(((g / S) & 1) ^ 1), abort_flag, p.err)) {
                    stop = true;
                    break;
                }
                const uint32_t st = smem_u32(smem + (size_t)s * p.stage_bytes);
                const uint32_t fb = bar_full + 8 * s;
                mbar_expect_tx(fb, p.tx_bytes);
                const int k0 = q * KVS;
                const uint32_t sb = st + (uint32_t)p.pieces * A_BYTES;
                tma_load_2d(st, &mA0, fb, k0, arow);
                tma_load_2d(sb, &mP0, fb, k0, prow);
                if (p.pieces > 1) {
                    tma_load_2d(st + A_BYTES, &mA1, fb, k0, arow);
                    tma_load_2d(sb + p.b_bytes, &mP1, fb, k0, prow);
                }
                if (p.pieces > 2) {
                    tma_load_2d(st + 2 * A_BYTES, &mA2, fb, k0, arow);
                    tma_load_2d(sb + 2 * p.b_bytes, &mP2, fb, k0, prow);
                }
                s_issued = g + 1;
            }
        }
    } else if (warp == pk::WARP_MMA && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = BF16 ? idesc_bf16(BM, p.bn) : idesc_tf32(BM, p.bn);
        const uint64_t desc0 = sdesc_sw128(smem_u32(smem));  // stage 0, piece 0
        int g = 0, gk = 0, j = 0;  // stages, k-blocks, tiles of this CTA so far
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++j) {
            for (int q = 0; q < nst; ++q, ++g) {
                const int s = g % S;
                const bool first = q % SPD == 0, last = q % SPD == SPD - 1 || q == nst - 1;  // of the k-block
                const int a = gk % nkb;
                if (!mbar_wait(bar_full + 8 * s, (uint32_t)((g / S) & 1), abort_flag, p.err) ||
                    (first && gk >= nkb &&
                     !mbar_wait(bar_kb_empty + 8 * a, (uint32_t)(((gk / nkb) - 1) & 1), abort_flag, p.err))) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)a * pk::KB_COLS;
                const uint32_t dc = ACC ? tmem + corr0 : d;  // correction products
                // operand descriptors by offset from the stage's first one (see the one-tile kernel)
                const uint64_t dA0 = desc0 + (uint64_t)(s * (p.stage_bytes >> 4));
                const uint64_t dA1 = dA0 + (A_BYTES >> 4);
                const uint64_t dB0 = dA0 + (uint64_t)(p.pieces * (A_BYTES >> 4));
                const uint64_t dB1 = dB0 + (p.b_bytes >> 4);
#pragma unroll
                for (int kk = 0; kk < KK; ++kk) {
                    const uint64_t o = 2 * kk;
                    mma_op<BF16>(d, dA0 + o, dB0 + o, idesc, (first && kk == 0) ? 0u : 1u);
                    if (!ACC && p.products >= 3) {  // ACC: the correction thread (below)
                        mma_op<BF16>(dc, dA1 + o, dB0 + o, idesc, 1u);
                        mma_op<BF16>(dc, dA0 + o, dB1 + o, idesc, 1u);
                    }
                }
                mma_commit(bar_empty + 8 * s);
                if (last) {
                    mma_commit(bar_kb_full + 8 * a);
                    ++gk;
                }
                s_consumed = g + 1;
            }
        }
        mma_commit(bar_done);
    } else if (ACC && warp == pk::WARP_MMA2 && lane == 0) {
        // ---------------- ACC: correction products into their own accumulator ----------------
        // A second issuing thread (one thread cannot issue 4 hi*hi and 20
        // correction products of 128 x 128 x 16 per k-block as fast as the tensor
        // core runs them). Its commits cover its own products: the stage's
        // `empty` (with the hi*hi thread's) and, after a tile's last stage,
        // corr_full, on which the drain warps wait before reading the region.
        const uint32_t idesc = BF16 ? idesc_bf16(BM, p.bn) : idesc_tf32(BM, p.bn);
        const uint64_t desc0 = sdesc_sw128(smem_u32(smem));
        const uint32_t dc = tmem + corr0;
        int g = 0, j = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++j) {
            for (int q = 0; q < nst; ++q, ++g) {
                const int s = g % S;
                if (!mbar_wait(bar_full + 8 * s, (uint32_t)((g / S) & 1), abort_flag, p.err) ||
                    (q == 0 && j > 0 && !mbar_wait(bar_corr_empty, (uint32_t)((j - 1) & 1), abort_flag, p.err))) {
                    stop = true;  // (or the previous tile's corrections were never read)
                    break;
                }
                tc_fence_after();
                const uint64_t dA0 = desc0 + (uint64_t)(s * (p.stage_bytes >> 4));
                const uint64_t dA1 = dA0 + (A_BYTES >> 4), dA2 = dA0 + 2 * (A_BYTES >> 4);
                const uint64_t dB0 = dA0 + (uint64_t)(p.pieces * (A_BYTES >> 4));
                const uint64_t dB1 = dB0 + (p.b_bytes >> 4), dB2 = dB0 + 2 * (p.b_bytes >> 4);
#pragma unroll
                for (int kk = 0; kk < KK; ++kk) {
                    const uint64_t o = 2 * kk;
                    if (p.products >= 3) {  // the tile's first correction product overwrites the region
                        mma_op<BF16>(dc, dA1 + o, dB0 + o, idesc, (q > 0 || kk > 0) ? 1u : 0u);
                        mma_op<BF16>(dc, dA0 + o, dB1 + o, idesc, 1u);
                    }
                    if (p.products == 6) {
                        mma_op<BF16>(dc, dA1 + o, dB1 + o, idesc, 1u);
                        mma_op<BF16>(dc, dA2 + o, dB0 + o, idesc, 1u);
                        mma_op<BF16>(dc, dA0 + o, dB2 + o, idesc, 1u);
                    }
                }
                mma_commit(bar_empty + 8 * s);
                if (q == nst - 1) mma_commit(bar_corr_full);
            }
        }
        mma_commit(bar_done);
    } else if (warp < pk::NUM_DRAIN) {
        // ---------------- drain: k-block sums -> FP32 register sums -> TMEM staging ----------------
        const int quarter = warp & 3, half = warp >> 2;
        const int hcols = p.bn / 2;  // 16, 32, 48 or 64 columns per warp
        const uint32_t lane_off = ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * hcols);
        int g = 0, j = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++j) {
            float sum[pk::HALF];
#pragma unroll
            for (int i = 0; i < pk::HALF; ++i) sum[i] = 0.f;
            for (int kb = 0; kb < nk; ++kb, ++g) {
                const int a = g % nkb;
                if (!warp_wait(bar_kb_full + 8 * a, (uint32_t)((g / nkb) & 1), abort_flag, p.err)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const uint32_t src = tmem + lane_off + (uint32_t)a * pk::KB_COLS;
#pragma unroll
                for (int c = 0; c < pk::HALF / 16; ++c) {
                    if (c * 16 < hcols) {
                        uint32_t r[16];
                        tmem_ld16(src + (uint32_t)(c * 16), r);
                        tmem_wait16(r);
#pragma unroll
                        for (int i = 0; i < 16; ++i) sum[c * 16 + i] += __uint_as_float(r[i]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_kb_empty + 8 * a);
            }
            if (stop) break;
            if constexpr (ACC) {
                // the correction thread's products of this tile have completed:
                // add the corrections, free the region
                if (!warp_wait(bar_corr_full, (uint32_t)(j & 1), abort_flag, p.err)) break;
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < pk::HALF / 16; ++c) {
                    if (c * 16 < hcols) {
                        uint32_t r[16];
                        tmem_ld16(tmem + lane_off + corr0 + (uint32_t)(c * 16), r);
                        tmem_wait16(r);
#pragma unroll
                        for (int i = 0; i < 16; ++i) sum[c * 16 + i] += __uint_as_float(r[i]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_corr_empty);
            }
            const int sb = j % nsb;
            if (j >= nsb && !warp_wait(bar_st_empty + 8 * sb, (uint32_t)(((j / nsb) - 1) & 1), abort_flag, p.err))
                break;
            tc_fence_after();
            const uint32_t dst = tmem + lane_off + staging0 + (uint32_t)sb * pk::KB_COLS;
#pragma unroll
            for (int c = 0; c < pk::HALF / 32; ++c) {
                if ((c + 1) * 32 <= hcols) {
                    uint32_t r[32];
#pragma unroll
                    for (int i = 0; i < 32; ++i) r[i] = __float_as_uint(sum[c * 32 + i]);
                    tmem_st32(dst + (uint32_t)(c * 32), r);
                } else if (c * 32 + 16 <= hcols) {
                    uint32_t r[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) r[i] = __float_as_uint(sum[c * 32 + i]);
                    tmem_st16(dst + (uint32_t)(c * 32), r);
                }
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_st_full + 8 * sb);
        }
    } else if (warp < pk::NUM_DRAIN + pk::NUM_STORE) {
        // ---------------- store warps: staging -> fused epilogue -> global ----------------
        // warp (quarter, half): TMEM lanes 32 quarter .. +31, columns half * bn/2 .. +bn/2
        const int quarter = warp & 3, half = (warp - pk::NUM_DRAIN) >> 2;
        const int hcols = p.bn / 2;
        constexpr int EC = pk::EPI_COLS;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            int tm, tn;
            tile_coords(t, p.tiles_m, p.tiles_n, 12, tm, tn);
            const int sb = j % nsb;
            if (!warp_wait(bar_st_full + 8 * sb, (uint32_t)((j / nsb) & 1), abort_flag, p.err)) break;
            tc_fence_after();
            const uint32_t src =
                tmem + ((uint32_t)(quarter * 32) << 16) + staging0 + (uint32_t)sb * pk::KB_COLS + (uint32_t)(half * hcols);
            const int grow = tm * BM + quarter * 32 + lane;  // row of the stacked components
            const bool row_ok = grow < p.nbatch * p.M;
            const int b = grow / p.M, mm = grow - b * p.M;
            const int mh = mm / p.n, ml = mm - mh * p.n;
            const int nn0 = tn * p.bn + half * hcols;
            const int cols = min(hcols, p.n - nn0);  // may be <= 0 for the last column tile
            if constexpr (VEC) {
                // the batch's 32 rows x EC columns go through shared memory so that
                // lane -> column cc, rows rr0 .. rr0+7: 16-byte accesses along the rows
                float* buf = s_epi + (warp - pk::NUM_DRAIN) * (EC * pk::EPI_CS);
                const int cc = lane >> 2, rr0 = (lane & 3) * 8;
                const int grow0 = tm * BM + quarter * 32 + rr0;
                const bool ok0 = grow0 < p.nbatch * p.M;
                const int b0 = ok0 ? grow0 / p.M : 0, mm0 = grow0 - b0 * p.M;
                const int mh0 = ok0 ? mm0 / p.n : 0, ml0 = mm0 - mh0 * p.n;
                float4 cur4[4], nxt4[4];
                if (ok0 && cc < cols) epi_load_rows8(p.e, b0, mh0, ml0, nn0 + cc, cur4);
                for (int c0 = 0; c0 < hcols; c0 += EC) {
                    uint32_t r[EC];
                    tmem_ld8(src + (uint32_t)c0, r);
                    const int c = c0 + cc;
                    if (ok0 && c + EC < cols) epi_load_rows8(p.e, b0, mh0, ml0, nn0 + c + EC, nxt4);
                    tmem_wait8(r);
#pragma unroll
                    for (int i = 0; i < EC; ++i) buf[i * pk::EPI_CS + lane] = __uint_as_float(r[i]);
                    __syncwarp();
                    const float4 a0 = *reinterpret_cast<const float4*>(buf + cc * pk::EPI_CS + rr0);
                    const float4 a1 = *reinterpret_cast<const float4*>(buf + cc * pk::EPI_CS + rr0 + 4);
                    __syncwarp();
                    if (ok0 && c < cols) {
                        const float v[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                        epi_apply_rows8(p.e, b0, mh0, ml0, nn0 + c, v, cur4);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) cur4[i] = nxt4[i];
                }
            } else {
            // state loads of the next EC columns go out before this batch's stores
            float2 cur[EC], nxt[EC];
            if (row_ok && cols > 0) epi_load_state<EC>(p.e, b, mh, ml, nn0, min(EC, cols), cur);
            for (int c0 = 0; c0 < hcols; c0 += EC) {
                uint32_t r[EC];
                tmem_ld8(src + (uint32_t)c0, r);
                if (row_ok && c0 + EC < cols)
                    epi_load_state<EC>(p.e, b, mh, ml, nn0 + c0 + EC, min(EC, cols - c0 - EC), nxt);
                tmem_wait8(r);
                if (row_ok && c0 < cols) {
                    float v[EC];
#pragma unroll
                    for (int i = 0; i < EC; ++i) v[i] = __uint_as_float(r[i]);
                    epi_apply_batch<EC>(p.e, b, mh, ml, nn0 + c0, v, min(EC, cols - c0), cur);
                }
#pragma unroll
                for (int i = 0; i < EC; ++i) cur[i] = nxt[i];
            }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_st_empty + 8 * sb);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == pk::WARP_TMA && lane == 0) {
        if (*abort_flag) {
            for (int g = s_consumed; g < s_issued; ++g) {
                const int s = g % S;
                const unsigned long long t0 = globaltimer();
                while (!mbar_try(bar_full + 8 * s, (uint32_t)((g / S) & 1)) && globaltimer() - t0 < 100000000ull) {
                }
            }
        }
        const unsigned long long t0 = globaltimer();
        while (!mbar_try(bar_done, 0u) && globaltimer() - t0 < 200000000ull) {
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == pk::WARP_TMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(pk::TMEM_COLS)
                     : "memory");
    }
}

// Diagnostic: one thread waits, through mbar_wait, on an mbarrier that no one
// arrives at, so the bounded wait runs out after limit_ns and raises ERR_TIMEOUT
// exactly as a stalled pipeline would; the kernel then returns normally.
__global__ void wait_timeout_probe_kernel(unsigned* err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_wait(smem_u32(&bar), 0u, &abort_flag, err, limit_ns);
    }
}

bool make_map(CUtensorMap* map, const void* base, int inner, long long rows, int ld, int box_rows, bool bf16) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) {
        snprintf(g_driver_error, sizeof g_driver_error, "cuTensorMapEncodeTiled entry point not found");
        return false;
    }
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * (bf16 ? 2 : 4)};
    cuuint32_t box[2] = {(cuuint32_t)(ROW / (bf16 ? 2 : 4)), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, ROW == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_driver_error, sizeof g_driver_error, "cuTensorMapEncodeTiled failed (%d) inner=%d rows=%lld ld=%d",
                 (int)r, inner, rows, ld);
        return false;
    }
    return true;
}

}  // namespace

const char* tc_last_driver_error() { return g_driver_error; }

namespace {

// Tile width: the multiple of 32 up to bn_max that wastes the fewest columns
// (each of the two column halves is a whole number of 16-column TMEM loads).
int pick_bn(int n, int bn_max) {
    if (n <= bn_max) return ((n + 31) / 32) * 32;
    int best = bn_max, best_waste = 1 << 30;
    for (int bn = bn_max; bn >= (bn_max > 128 ? 128 : 64); bn -= 32) {
        const int waste = ((n + bn - 1) / bn) * bn - n;
        if (waste < best_waste) {
            best_waste = waste;
            best = bn;
        }
    }
    return best;
}

int pieces_of(int products) { return products == 6 ? 3 : (products == 3 ? 2 : 1); }

// Can the persistent kernel run this pass? Its accurate variant has no
// compensated sums across k-blocks, so it takes short K ranges only (at most
// 16 k-blocks); its fast variant reads at most two operand pieces.
bool persistent_ok(int n, int pieces, bool accurate, bool bf16) {
    const int kv = bf16 ? 2 * BKF : BKF;
    const int nk = (n + kv - 1) / kv;
    return accurate ? nk <= 16 : pieces <= 2;
}

// The largest tile width the one-tile kernel takes: 128 for the accurate
// variant (its epilogue holds two sums per column) and for three pieces (a
// 128 x 256 tile of three pieces leaves room for one pipeline stage).
int onetile_bn_max(int pieces, bool accurate) { return (accurate || pieces == 3) ? 128 : 256; }

TcConfig tc_make(int M, int n, int products, int nbatch, bool bf16, bool accurate, bool persistent, int bn) {
    TcConfig c{};
    c.products = products;
    c.bf16 = bf16;
    c.pieces = pieces_of(products);
    c.accurate = accurate && c.pieces >= 2;
    c.persistent = persistent;
    const long long rows = (long long)nbatch * M;  // components / instances stacked
    c.bn = bn;
    c.tiles_n = (n + c.bn - 1) / c.bn;
    c.tiles_m = (int)((rows + BM - 1) / BM);
    const unsigned b_bytes = (unsigned)c.bn * ROW;
    c.stage_bytes = (unsigned)c.pieces * ((unsigned)A_BYTES + b_bytes);
    // the persistent kernel's static shared memory (transposition buffers) comes off the ring
    int s = (SMEM_LIMIT - 1024 - (persistent ? pk::STATIC_SMEM : 0)) / (int)c.stage_bytes;
    if (s > 8) s = 8;
    if (c.persistent) {
        c.tmem_cols = (int)pk::TMEM_COLS;  // k-block buffers, corrections / staging buffers of 128 columns
    } else {
        int acc = 32;
        while (acc < c.bn) acc *= 2;
        // two k-block accumulator buffers (+ the correction accumulator in ACCURATE
        // mode), rounded up to the power of two that tcgen05.alloc needs
        c.tmem_cols = c.accurate ? 4 * acc : 2 * acc;
        // the epilogue stages 8 warps x 32 rows x MAX_HALF sums in the pipeline buffers
        while (s * (int)c.stage_bytes < STAGE_BYTES_EPI && (s + 1) * (int)c.stage_bytes <= SMEM_LIMIT - 1024) ++s;
    }
    c.stages = s;
    c.smem_bytes = s * (int)c.stage_bytes + 1024;
    return c;
}

}  // namespace

TcConfig tc_choose(int M, int n, int products, int nbatch, bool bf16, bool accurate) {
    const int pieces = pieces_of(products);
    accurate = accurate && pieces >= 2;
    // The 128 x 256 one-tile-per-CTA kernel wins when each tile has a long K loop
    // and there are enough tiles to fill the SMs several times over (2D at large
    // n); otherwise (3D: K = n is short, the epilogue dominates; mid-size 2D:
    // few tiles) the persistent 128 x 128 kernel overlaps epilogue and products.
    const int kv = bf16 ? 2 * BKF : BKF;
    const int nk = (n + kv - 1) / kv;
    const long long rows = (long long)nbatch * M;
    const long long tiles256 = ((rows + BM - 1) / BM) * ((n + 255) / 256);
    const bool long_k = nk * kv >= 2048 && tiles256 >= 4 * 152;
    const bool persistent = !long_k && persistent_ok(n, pieces, accurate, bf16);
    const int bn = pick_bn(n, persistent ? 128 : onetile_bn_max(pieces, accurate));
    return tc_make(M, n, products, nbatch, bf16, accurate, persistent, bn);
}

int tc_candidates(int M, int n, int products, int nbatch, bool bf16, bool accurate, TcConfig* out, int max_out) {
    const int pieces = pieces_of(products);
    accurate = accurate && pieces >= 2;
    TcConfig c[4];
    int k = 0;
    c[k++] = tc_choose(M, n, products, nbatch, bf16, accurate);
    const int bmax = onetile_bn_max(pieces, accurate);
    c[k++] = tc_make(M, n, products, nbatch, bf16, accurate, false, pick_bn(n, bmax));
    if (bmax > 128) c[k++] = tc_make(M, n, products, nbatch, bf16, accurate, false, pick_bn(n, 128));
    if (persistent_ok(n, pieces, accurate, bf16))
        c[k++] = tc_make(M, n, products, nbatch, bf16, accurate, true, pick_bn(n, 128));
    int m = 0;
    for (int i = 0; i < k && m < max_out; ++i) {
        bool dup = false;
        for (int j = 0; j < m; ++j) dup = dup || (out[j].persistent == c[i].persistent && out[j].bn == c[i].bn);
        if (!dup) out[m++] = c[i];
    }
    return m;
}

cudaError_t tc_maps_create(TcMaps** out, int M, int n, int nbatch, int ld, const void* const a[][3], int n_a,
                           const void* const pp[3], const int bn_slot[2], bool bf16) {
    *out = nullptr;
    if (n_a > 4) return cudaErrorInvalidValue;
    TcMaps* m = new TcMaps();
    m->n_a = n_a;
    bool ok = true;
    for (int i = 0; i < n_a && ok; ++i)
        for (int j = 0; j < 3 && ok; ++j) {
            const void* base = a[i][j] ? a[i][j] : a[i][0];
            ok = make_map(&m->a[i][j], base, n, (long long)nbatch * M, ld, BM, bf16);
        }
    for (int slot = 0; slot < 2 && ok; ++slot)
        for (int j = 0; j < 3 && ok; ++j) {
            const void* base = pp[j] ? pp[j] : pp[0];
            ok = make_map(&m->p[slot][j], base, n, n, ld, bn_slot[slot] > 0 ? bn_slot[slot] : 32, bf16);
        }
    if (!ok) {
        delete m;
        return cudaErrorInvalidValue;
    }
    static bool attr_set = false;
    if (!attr_set) {
        const void* kernels[12] = {(const void*)gemm_tf32_tc_kernel<false, false>,
                                 (const void*)gemm_tf32_tc_kernel<true, false>,
                                 (const void*)gemm_tf32_tc_kernel<false, true>,
                                 (const void*)gemm_tf32_tc_kernel<true, true>,
                                 (const void*)gemm_tf32_persistent_kernel<false, false, false>,
                                 (const void*)gemm_tf32_persistent_kernel<true, false, false>,
                                 (const void*)gemm_tf32_persistent_kernel<false, true, false>,
                                 (const void*)gemm_tf32_persistent_kernel<true, true, false>,
                                 (const void*)gemm_tf32_persistent_kernel<false, false, true>,
                                 (const void*)gemm_tf32_persistent_kernel<true, false, true>,
                                 (const void*)gemm_tf32_persistent_kernel<false, true, true>,
                                 (const void*)gemm_tf32_persistent_kernel<true, true, true>};
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < 12; ++i)  // persistent kernels (4-11): room for the VEC transposition buffers
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kernels[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         i < 4 ? SMEM_LIMIT : SMEM_LIMIT - (pk::STATIC_SMEM - 1024));
        if (e != cudaSuccess) {
            delete m;
            return e;
        }
        attr_set = true;
    }
    *out = m;
    return cudaSuccess;
}

void tc_maps_destroy(TcMaps* m) { delete m; }

cudaError_t launch_wait_timeout_probe(unsigned* err, double limit_ms, cudaStream_t st) {
    wait_timeout_probe_kernel<<<1, 32, 0, st>>>(err, (unsigned long long)(limit_ms * 1e6));
    return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const TcConfig& cfg, int slot, const TcMaps* maps, int a_index, int M, int n, int nbatch,
                           const Epi<float>& e, unsigned* err, cudaStream_t st) {
    if (a_index < 0 || a_index >= maps->n_a || slot < 0 || slot > 1) return cudaErrorInvalidValue;
    KParams p;
    p.M = M;
    p.n = n;
    p.bn = cfg.bn;
    p.stages = cfg.stages;
    p.products = cfg.products;
    p.pieces = cfg.pieces;
    p.tiles_m = cfg.tiles_m;
    p.tiles_n = cfg.tiles_n;
    p.tmem_cols = cfg.tmem_cols;
    p.acc_cols = cfg.tmem_cols / (cfg.accurate ? 4 : 2);
    p.stage_bytes = cfg.stage_bytes;
    p.b_bytes = (unsigned)cfg.bn * ROW;
    p.tx_bytes = cfg.stage_bytes;
    p.err = err;
    p.e = e;
    p.nbatch = nbatch;
    p.vec = epi_rows8_ok(e) ? 1 : 0;
    const long long ntiles = (long long)cfg.tiles_m * cfg.tiles_n;
    const CUtensorMap* A = maps->a[a_index];
    const CUtensorMap* P = maps->p[slot];
    if (cfg.persistent) {
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
        }
        const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
        const int sm = cfg.smem_bytes;
        const int th = pk::THREADS;
#define ETD_PK(B, C, V) gemm_tf32_persistent_kernel<B, C, V><<<grid, th, sm, st>>>(A[0], A[1], A[2], P[0], P[1], P[2], p)
        if (p.vec) {
            if (cfg.accurate && cfg.bf16) ETD_PK(true, true, true);
            else if (cfg.accurate) ETD_PK(false, true, true);
            else if (cfg.bf16) ETD_PK(true, false, true);
            else ETD_PK(false, false, true);
        } else {
            if (cfg.accurate && cfg.bf16) ETD_PK(true, true, false);
            else if (cfg.accurate) ETD_PK(false, true, false);
            else if (cfg.bf16) ETD_PK(true, false, false);
            else ETD_PK(false, false, false);
        }
#undef ETD_PK
    } else {
        const unsigned g = (unsigned)ntiles;
        const int sm = cfg.smem_bytes;
        if (cfg.accurate && cfg.bf16)
            gemm_tf32_tc_kernel<true, true><<<g, NUM_THREADS, sm, st>>>(A[0], A[1], A[2], P[0], P[1], P[2], p);
        else if (cfg.accurate)
            gemm_tf32_tc_kernel<true, false><<<g, NUM_THREADS, sm, st>>>(A[0], A[1], A[2], P[0], P[1], P[2], p);
        else if (cfg.bf16)
            gemm_tf32_tc_kernel<false, true><<<g, NUM_THREADS, sm, st>>>(A[0], A[1], A[2], P[0], P[1], P[2], p);
        else
            gemm_tf32_tc_kernel<false, false><<<g, NUM_THREADS, sm, st>>>(A[0], A[1], A[2], P[0], P[1], P[2], p);
    }
    return cudaGetLastError();
}

}  // namespace etd
