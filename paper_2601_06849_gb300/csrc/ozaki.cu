// FP64-split transform pass (ETD_PREC_FP64_SPLIT): the dense product with P of
// Section 3.3.2 in FP64 accuracy on the BF16 tensor cores, by error-free
// splitting into integer slices (the splitting scheme of Ozaki et al. for
// accurate matrix products on low-precision units).
//
//     out(b, mm, nn) = sum_k A[b][mm][k] P[nn][k]          (FP64 fields, FP64 result)
//
// Slices. Every operand value x of row r (the n values one output row contracts)
// is written as a fixed-point number below the power of two 2^e_r > max |x| over the row:
//     x ~ 2^(e_r - 48) t,   t = round(x 2^(48 - e_r)),  |t| <= 2^48,
// and t is cut into OZ_S = 6 balanced base-256 digits, most significant first,
//     t = sum_i a_i 2^(8 (5 - i)),   a_1 .. a_5 in [-128, 128],  |a_0| <= 256.
// P is cut the same way below its own scale 2^e_P > max |P| (about sqrt(2/(n+1)):
// a fixed scale of 1 would leave its top slices nearly empty), once per plan on
// the host, with one bit less (t_P = round(p 2^(47 - e_P)), so |p_0| <= 128 too).
// Every slice is an integer of at most 8 significant bits, exact in BF16; a slice
// product is at most 2^15 in magnitude when it involves a_0, else 2^14. Balanced
// digits carry 8 bits of the value in a slice of magnitude 2^7: the product bound
// of 7-bit slices with the information of 8-bit ones.
//
// Products. The product of slices a_i and p_j carries the weight 2^(-8 (i + j));
// all pairs (i, j) of one level l = i + j <= 5 (21 pairs) accumulate in one TMEM
// accumulator over a group of OZ_GROUP = 4 k-blocks of 32 values: at most
// (2^15 + l 2^14) x 128 <= 7 x 2^21 < 2^24 in magnitude, so the FP32 accumulation
// of these integers is exact whatever the order of the additions inside the
// tensor core. The group sums S_l are added in int32 registers (exact up to
// K = 16384: 128 groups x 7 x 2^21 < 2^31), and at the end
//     out = 2^(e_r + e_P - 55) (J 2^16 + H_2),   J = H_0 2^16 + H_1,
//     H_g = S_2g 2^8 + S_2g+1                     (int64, exact)
// is formed in FP64 (one rounding while |J| < 2^46, else two). What is left out: the rounding of each
// operand to 48 bits below its row's scale (2^-49 relative to the row's max; P:
// 2^-48) and the pairs with i + j >= 6 (each below 2^-49 of the scales' product
// per term, of random sign): a few 2^-48 relative to the row's max |out|. The
// scale is per row, not per component: the spectral coefficients of a field
// dominated by a constant (FitzHugh-Nagumo's v, driven by eps b) are large in a
// few modes, and the back-transform recovers the field through heavy
// cancellation; with one scale per component that lost 40x more (CPU emulation
// of this arithmetic, n = 512: 7.3e-11 against 1.9e-12). The small slices are
// what allows a TMEM buffer to accumulate four k-blocks before it is drained: the
// drain (TMEM loads, int32 sums) bounded the kernel when it ran after every
// k-block (unbalanced 8-bit slices, products up to 2^16).
//
// Fewer slices (ETD_PREC_FP64_SPLIT40: S = 5, ETD_PREC_FP64_SPLIT32: S = 4): the
// same scheme with t rounded to 8S bits (P: 8S - 1), S digits, levels l <= S - 1
// (S (S + 1) / 2 pairs), out = 2^(e_r + e_P - 8S - 7) sum_l S_l 2^(8 (S - 1 - l)),
// and smaller pipeline stages (more of them in flight); the kernels below are
// templates on S.
//
// Per pass: a slicing kernel (one warp per operand row, one block per row for rows
// of more than 1024 values: the row's scale, then its S BF16 slices, written into
// tiled planes: 128 rows x 32 values per tile, contiguous and already in the
// swizzled order of the shared-memory stage) and
// the product kernel, persistent (one CTA per SM walks the 128 x 32 tiles; the MMA
// warp fills the two TMEM buffers with the next tile's first groups while the
// drain warps run the previous tile's epilogue):
//   warps 0-15 drain: per group of four k-blocks, tcgen05.ld of the S level
//              accumulators of their TMEM lane quarter and 8-column quarter (two
//              levels per load round trip), integer sums; at the end the FP64
//              result and the fused epilogue (Epi<double>, the Hadamard stages
//              and outputs of the FP64 path);
//   warp 16    TMA producer (one lane: per k-block twelve untiled bulk copies,
//              one contiguous tile of each slice plane of A (8 KB) and of P
//              (2 KB); a 2D tensor map would fetch the same bytes as 64-byte
//              rows, twice the requests) and TMEM allocator;
//   warp 17    MMA issuer (one lane): per k-step of 16 values, one product per A
//              slice i with all P slices j <= 5 - i at once. The six level
//              accumulators of a buffer are consecutive 32-column TMEM blocks and
//              the P slices consecutive 32-row blocks of shared memory, so the
//              product of A slice i (M = 128, K = 16) with P slices 0 .. 5 - i
//              (N = 32 (6 - i)), written from level block i on, adds a_i p_j to
//              level block i + j: 6 products per k-step instead of 21, each A
//              chunk read from shared memory once per k-step.
// (Products, levels and stages as written for S = 6.) Shared memory holds three
// pipeline stages of 32 K-values (64-byte rows, 64-byte swizzle) of the six A
// slices and the six P slices (60 KB per stage; S = 5, 4: four stages of 50 KB,
// five of 40 KB). TMEM holds two buffers of S 32-column level accumulators.
// Every wait is bounded (tc_ptx.cuh); on expiry the CTA raises ERR_TIMEOUT and
// returns after its copies and products have completed (bounded as well).
#include <cuda.h>
#include <stdio.h>

#include "etd_internal.cuh"
#include "tc_ptx.cuh"

namespace etd {

namespace {

constexpr int OZ_BM = OZ_TILE_ROWS_A;
constexpr int OZ_BN = OZ_TILE_ROWS_P;
static_assert(OZ_BM == 1 << 7 && OZ_BN == 1 << 5, "the tile offsets below take 128-row A and 32-row P tiles");
constexpr int OZ_KV = 32;   // BF16 values of K per pipeline stage (one k-block)
constexpr int OZ_ROW = 64;  // bytes of K per operand row in a stage
constexpr int OZ_A_BYTES = OZ_BM * OZ_ROW;
constexpr int OZ_B_BYTES = OZ_BN * OZ_ROW;
// Per slice count S (6: ETD_PREC_FP64_SPLIT, 5: _SPLIT40, 4: _SPLIT32): bytes of one
// pipeline stage, stages that fit (3 x 60 KB, 4 x 50 KB, 5 x 40 KB), dynamic shared memory.
__host__ __device__ constexpr int oz_stage_bytes(int S) { return S * (OZ_A_BYTES + OZ_B_BYTES); }
__host__ __device__ constexpr int oz_stages(int S) { return S == 6 ? 3 : (S == 5 ? 4 : 5); }
__host__ __device__ constexpr int oz_smem(int S) { return oz_stages(S) * oz_stage_bytes(S) + 1024; }  // + alignment
constexpr int OZ_DRAIN_WARPS = 16;                   // four per TMEM lane quarter
constexpr int OZ_DC = OZ_BN * 4 / OZ_DRAIN_WARPS;   // columns of a tile per drain warp (8)
constexpr int OZ_WARP_TMA = OZ_DRAIN_WARPS;
constexpr int OZ_WARP_MMA = OZ_DRAIN_WARPS + 1;
constexpr int OZ_THREADS = (OZ_DRAIN_WARPS + 2) * 32;
static_assert(OZ_DC == 8, "the drain loads eight columns per level (tcgen05.ld 32x32b.x8)");
constexpr uint32_t OZ_TMEM_COLS = 512;  // 2 buffers x S levels x 32 columns (at most 384), allocated as 512
constexpr int OZ_BITS = 8;
// bits below an operand row's scale (8 S: 48, 40 or 32); P takes one bit less, so that
// its top slice stays within 128
__host__ __device__ constexpr int oz_frac(int S) { return S * OZ_BITS; }
constexpr int OZ_GROUP = 4;              // k-blocks (32 values each) a TMEM buffer accumulates before a drain
static_assert(2 * OZ_S * OZ_BN <= (int)OZ_TMEM_COLS, "level accumulators exceed the TMEM allocation");
static_assert(oz_smem(6) <= 227 * 1024 && oz_smem(5) <= 227 * 1024 && oz_smem(4) <= 227 * 1024,
              "pipeline stages exceed the shared memory of a CTA");

struct OzPlanes {
    __nv_bfloat16* s[OZ_S];
};

struct OzParams {
    const uint8_t* a[OZ_S];  // the operand's slice planes, tiles of OZ_BM rows x 32 values
    const uint8_t* b[OZ_S];  // P's slice planes, tiles of OZ_BN rows x 32 values
    int nkb;                 // k-blocks of 32 values per row: ceil(n / 32)
    int M, n, nbatch, tiles_m, tiles_n;
    int p_exp;                       // P's scale exponent e_P
    const int* rexp;                 // per row of the stacked entries: its scale exponent or code
    unsigned* err;
    Epi<double> e;
};

// 2^k as a double, for -1022 <= k <= 1023 (built from its bits: exact, no libm).
__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Row exponent codes besides a finite scale exponent (|e| < 1100).
constexpr int OZ_EXP_ZERO = -4096;       // row of zeros: zero slices, zero result
constexpr int OZ_BEXP_MIN = 193;         // rows with max |x| < 2^-830 count as zero rows

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
constexpr int OZ_EXP_NONFINITE = 4096;   // row with NaN or Inf: NaN result

// Untiled bulk copy of `bytes` contiguous bytes from global to shared memory,
// completing on the mbarrier at `bar` (both addresses 16-byte aligned, bytes a
// multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace

// Element offset of value k of row r in a tiled slice plane. A plane is a
// sequence of tiles of 2^rows_log2 rows x 32 values (64-byte rows), ordered by
// (row block, k-block); inside a tile the 16-byte chunk c of row rr sits at chunk
// c ^ ((rr >> 1) & 3): the 64-byte swizzle of the shared-memory operand layout
// the MMA reads. One untiled bulk copy then brings a tile into a 1024-byte
// aligned pipeline stage as it is. Values past n in the last k-block and rows
// past the last one stay zero (the planes are cleared once when allocated).
__host__ __device__ __forceinline__ long long oz_tile_off(long long r, int k, int nkb, int rows_log2) {
    const long long rb = r >> rows_log2;
    const int rr = (int)(r & ((1 << rows_log2) - 1));
    const int kb = k >> 5, kc = (k >> 3) & 3, e = k & 7;
    return ((rb * nkb + kb) << (rows_log2 + 5)) + rr * 32 + ((kc ^ ((rr >> 1) & 3)) << 3) + e;
}

namespace {

// FP64 arithmetic runs at about two operations per clock and SM on this GPU, 64
// times slower than FP32; the slicing is integer arithmetic on the bit patterns
// for the rounding and exact FP32 arithmetic for the digits instead (an
// integer-only forming of the result in the product kernel's epilogue measured
// slower than its four FP64 operations, and was dropped).
//
// q = round(|x| 2^(F - e)) to nearest, ties to even, for |x| < 2^e (F = 48, 40 or 32),
// from the bits of x: |x| = m 2^(b - 1075) (m with its implicit bit, b the biased
// exponent, 1 for a subnormal), so q = m 2^-sh with sh = 1075 - F + e - b >= 5.
template <int F>
__device__ __forceinline__ unsigned long long oz_round_mag(unsigned long long bits, int e) {
    const int b = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(b != 0) << 52);
    const int sh = 1075 - F + e - (b == 0 ? 1 : b);
    // floor((m + 2^(sh-1) - 1 + lsb) / 2^sh), lsb the last bit of floor(m / 2^sh):
    // ties go to the even quotient (m + 2^(sh-1) < 2^54: no overflow)
    return sh < 64 ? (m + ((1ull << (sh - 1)) - 1) + ((m >> sh) & 1)) >> sh : 0;
}

// rne(v / 256) for |v| < 2^30: adding 1.5 2^23 to |y| < 2^22 leaves a sum whose last
// place is 1, so the sum is y rounded to an integer (ties to even), and taking
// 1.5 2^23 off again is exact. Both operations are written with explicit rounding,
// so the compiler neither contracts nor cancels them.
constexpr float OZ_RND = 12582912.0f;
__device__ __forceinline__ float oz_rne_div256(float v) {
    return __fadd_rn(__fmaf_rn(v, 0.00390625f, OZ_RND), -OZ_RND);
}

// S balanced base-256 digits of t = sign(x) q (q <= 2^(8 S)). q is split once as
// q = hi 2^24 + lo with lo in [-2^23, 2^23) (two integer operations each), both
// converted exactly to FP32 with x's sign; each half is then cut in FP32 by
// u = rne(v / 256), digit v - 256 u (an exact fma: an integer of at most 8 bits),
// v <- u; the last quotient of each half is its top digit: |a_i| <= 128 below the
// top, |a_(S-3)| <= 128, |a_0| <= 256 (hi <= 2^24 has S - 3 digits). All values
// are integers below 2^25, so every operation is exact.
template <int S>
__device__ __forceinline__ void oz_digits(unsigned long long q, unsigned x_hi, float (&a)[OZ_S]) {
    static_assert(S >= 4 && S <= 6 && OZ_BITS == 8, "oz_digits is written for four to six balanced 8-bit slices");
    const unsigned q0 = (unsigned)q, q1 = (unsigned)(q >> 32);
    const int lo = (int)(q0 << 8) >> 8;                                  // low 24 bits of q, balanced
    const unsigned hi = __funnelshift_r(q0, q1, 24) + ((q0 >> 23) & 1u);  // (q - lo) / 2^24
    const float sg = __int_as_float((int)((x_hi & 0x80000000u) | 0x3F800000u));  // sign(x) as +-1
    const float lf = __fmul_rn((float)lo, sg), hf = __fmul_rn((float)hi, sg);
    const float u = oz_rne_div256(lf);
    a[S - 1] = __fmaf_rn(u, -256.f, lf);
    const float u2 = oz_rne_div256(u);
    a[S - 2] = __fmaf_rn(u2, -256.f, u);
    a[S - 3] = u2;
    if constexpr (S == 6) {
        const float v = oz_rne_div256(hf);
        a[2] = __fmaf_rn(v, -256.f, hf);
        const float v2 = oz_rne_div256(v);
        a[1] = __fmaf_rn(v2, -256.f, v);
        a[0] = v2;
    } else if constexpr (S == 5) {
        const float v = oz_rne_div256(hf);
        a[1] = __fmaf_rn(v, -256.f, hf);
        a[0] = v;
    } else {
        a[0] = hf;
    }
}

// Biased exponent field of x (0x7FF for NaN and Inf): the largest one over a row
// is the biased exponent of the row's max |x|.
__device__ __forceinline__ unsigned oz_bexp(double x) { return ((unsigned)__double2hiint(x) >> 20) & 0x7FFu; }

// A row's scale code from the biased exponent of its max |x|: e_r with
// max |x| < 2^e_r (frexp's exponent of the max); OZ_EXP_ZERO for a row of zeros (or
// max below 2^-830: its slices are zero), OZ_EXP_NONFINITE for a row with NaN or
// Inf (its first slice carries them, so the products and the result of the row are NaN).
__device__ __forceinline__ int oz_row_code(int bmax) {
    return bmax == 0x7FF ? OZ_EXP_NONFINITE : (bmax < OZ_BEXP_MIN ? OZ_EXP_ZERO : bmax - 1022);
}

// The S slices of one value x of a row with scale code `code`.
template <int S>
__device__ __forceinline__ void oz_cut_value(double x, int code, float (&a)[OZ_S]) {
    if (code == OZ_EXP_NONFINITE) {
#pragma unroll
        for (int i = 0; i < S; ++i) a[i] = 0.f;
        if ((abs_bits(x) >> 52) == 0x7FF) a[0] = (float)x;  // NaN / Inf into the products
    } else if (code == OZ_EXP_ZERO) {
#pragma unroll
        for (int i = 0; i < S; ++i) a[i] = 0.f;
    } else {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
        oz_digits<S>(oz_round_mag<oz_frac(S)>(bits, code), (unsigned)(bits >> 32), a);
    }
}

// Values 2k, 2k + 1 of a row (one 4-byte word of each plane, at element offset o).
template <int S>
__device__ __forceinline__ void oz_store_pair(const OzPlanes& out, long long o, double x0, double x1, int code) {
    float a[OZ_S], b[OZ_S];
    oz_cut_value<S>(x0, code, a);
    oz_cut_value<S>(x1, code, b);
#pragma unroll
    for (int i = 0; i < S; ++i)  // exact: integers of at most 8 significant bits
        *reinterpret_cast<__nv_bfloat162*>(out.s[i] + o) = __floats2bfloat162_rn(a[i], b[i]);
}

// The last value of a row of odd length n.
template <int S>
__device__ __forceinline__ void oz_store_last(const OzPlanes& out, long long r, int n, int nkb, double x, int code) {
    float a[OZ_S];
    oz_cut_value<S>(x, code, a);
    const long long o = oz_tile_off(r, n - 1, nkb, 7);
#pragma unroll
    for (int i = 0; i < S; ++i) out.s[i][o] = __float2bfloat16_rn(a[i]);
}

// The S BF16 slice planes of A (tiled, 128-row tiles) and each row's scale code
// rexp[r] (oz_row_code), one warp per row of the stacked batch entries (row r at
// r * ld; its n values are written, the tiles' padding stays zero): the warp
// reduces max |x| over the row, then cuts every value below 2^e_r > max |x| (the
// row is read again, from L1/L2 for rows of up to 1024 values).
template <int S>
__global__ void __launch_bounds__(256) oz_slice_kernel(const double* __restrict__ A, long long rows, int n, int ld,
                                                      int nkb, int* __restrict__ rexp, OzPlanes out) {
    const int lane = threadIdx.x & 31;
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    const int npair = n >> 1;  // value pairs per row (rows start on even elements: ld is a multiple of 8)
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += wstride) {
        const double* row = A + r * ld;
        const double2* row2 = reinterpret_cast<const double2*>(row);
        unsigned bx = 0;
        for (int k = lane; k < npair; k += 32) {
            const double2 v = row2[k];
            bx = max(bx, max(oz_bexp(v.x), oz_bexp(v.y)));
        }
        if ((n & 1) && lane == 0) bx = max(bx, oz_bexp(row[n - 1]));
        const int code = oz_row_code((int)__reduce_max_sync(0xffffffffu, bx));
        if (lane == 0) rexp[r] = code;
        // k + 32 lies two k-blocks (two tiles of 128 x 32 values) further on, at
        // the same place in its tile
        long long o = oz_tile_off(r, 2 * lane, nkb, 7);
        for (int k = lane; k < npair; k += 32, o += 2 * OZ_BM * OZ_KV) {
            const double2 v = row2[k];
            oz_store_pair<S>(out, o, v.x, v.y, code);
        }
        if ((n & 1) && lane == 0) oz_store_last<S>(out, r, n, nkb, row[n - 1], code);
    }
}

// The same slicing for rows of more than 1024 values: one block per row, each
// thread holding up to OZ_PT value pairs in registers from the max to the cut, so
// the row is read once. (With one warp per row of 4096 values, the rows in flight,
// 54 of 32 KB per SM, exceed the L2 and the second read came from DRAM.)
constexpr int OZ_PT = 8;
constexpr int OZ_SLICE_ROW_MIN = 1025;  // rows of at least this many values take the block-per-row kernel

__host__ __device__ constexpr int oz_slice_row_threads(int n) {  // a multiple of 32, at most 1024 for n <= 16384
    return 32 * (((n >> 1) + OZ_PT * 32 - 1) / (OZ_PT * 32));
}

template <int S>
__global__ void __launch_bounds__(1024) oz_slice_row_kernel(const double* __restrict__ A, int n, int ld, int nkb,
                                                          int* __restrict__ rexp, OzPlanes out) {
    __shared__ unsigned s_bx[32];
    const long long r = blockIdx.x;
    const double* row = A + r * ld;
    const double2* row2 = reinterpret_cast<const double2*>(row);
    const int npair = n >> 1, nt = blockDim.x, t = threadIdx.x;  // npair <= OZ_PT nt (launch rule)
    double2 v[OZ_PT];
    unsigned bx = 0;
#pragma unroll
    for (int j = 0; j < OZ_PT; ++j) {
        const int k = t + j * nt;
        v[j] = k < npair ? row2[k] : make_double2(0.0, 0.0);
        bx = max(bx, max(oz_bexp(v[j].x), oz_bexp(v[j].y)));
    }
    const double last = (n & 1) ? row[n - 1] : 0.0;
    bx = max(bx, oz_bexp(last));
    bx = __reduce_max_sync(0xffffffffu, bx);
    if ((t & 31) == 0) s_bx[t >> 5] = bx;
    __syncthreads();
    bx = 0;
    for (int w = 0; w < (nt >> 5); ++w) bx = max(bx, s_bx[w]);
    const int code = oz_row_code((int)bx);
    if (t == 0) rexp[r] = code;
    // pair k + nt lies 2 nt / 32 k-blocks further on, at the same place in its tile
    // (nt is a multiple of 16)
    long long o = oz_tile_off(r, 2 * t, nkb, 7);
    const long long step = (long long)(2 * nt / OZ_KV) * (OZ_BM * OZ_KV);
#pragma unroll
    for (int j = 0; j < OZ_PT; ++j, o += step)
        if (t + j * nt < npair) oz_store_pair<S>(out, o, v[j].x, v[j].y, code);
    if ((n & 1) && t == 0) oz_store_last<S>(out, r, n, nkb, last, code);
}

}  // namespace

namespace {

// The six-slice result (J 2^16 + H_2) 2^E: while |J| < 2^46 the sum is exact in
// int64 and takes one conversion, the scale going into the exponent field; the
// rest (large sums, results outside the normal range) takes the general form in
// a function of its own, so that the common path is not predicated with it.
__device__ __noinline__ double oz_form6_general(long long J, long long H2, double scale) {
    return fma((double)J, pow2(2 * OZ_BITS), (double)H2) * scale;
}
__device__ __forceinline__ double oz_form6(long long J, long long H2, int E, double scale) {
    if (J < (1ll << 46) && J > -(1ll << 46)) {
        const double v = (double)(J * 65536 + H2);
        const long long bits = __double_as_longlong(v);
        const int be = (int)((bits >> 52) & 0x7FF);
        if (be != 0 && be + E >= 1 && be + E <= 2046) return __longlong_as_double(bits + ((long long)E << 52));
    }
    return oz_form6_general(J, H2, scale);
}

template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1) ozaki_pass_kernel(const __grid_constant__ OzParams p) {
    constexpr int STAGES = oz_stages(S), STAGE_BYTES = oz_stage_bytes(S);
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_skip;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_consumed;
    __shared__ int s_issued;
    // full[3], empty[3] (shared-memory ring), acc_full[2], acc_empty[2] (TMEM ring), done
    __shared__ __align__(8) uint64_t s_bar[2 * STAGES + 5];

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) s_skip = (*(volatile unsigned*)p.err != 0u);
    __syncthreads();
    if (s_skip) return;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    volatile int* abort_flag = &s_abort;
    const uint32_t bar_full = smem_u32(&s_bar[0]);
    const uint32_t bar_empty = smem_u32(&s_bar[STAGES]);
    const uint32_t bar_acc_full = smem_u32(&s_bar[2 * STAGES]);
    const uint32_t bar_acc_empty = smem_u32(&s_bar[2 * STAGES + 2]);
    const uint32_t bar_done = smem_u32(&s_bar[2 * STAGES + 4]);

    const int nk = (p.n + OZ_KV - 1) / OZ_KV;  // k-blocks of a tile (one pipeline stage each)
    const int ng = (nk + OZ_GROUP - 1) / OZ_GROUP;  // k-block groups of a tile (one TMEM buffer each)
    const int ntiles = p.tiles_m * p.tiles_n;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(bar_acc_full + 8 * a, 1);
            mbar_init(bar_acc_empty + 8 * a, OZ_DRAIN_WARPS);
        }
        mbar_init(bar_done, 1);
        s_abort = 0;
        s_consumed = 0;
        s_issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == OZ_WARP_TMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(OZ_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == OZ_WARP_TMA && lane == 0) {
        // ---------------- TMA producer: the A and P slices of each k-block, tile after tile ----------------
        int gq = 0;  // k-blocks issued by this CTA so far (one ring across tiles)
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, p.tiles_m, p.tiles_n, 8, tm, tn);
            for (int q = 0; q < nk; ++q, ++gq) {
                const int s = gq % STAGES;
                if (!mbar_wait(bar_empty + 8 * s, (uint32_t)(((gq / STAGES) & 1) ^ 1), abort_flag, p.err)) {
                    stop = true;
                    break;
                }
                const uint32_t st = smem_u32(smem + (size_t)s * STAGE_BYTES);
                const uint32_t fb = bar_full + 8 * s;
                mbar_expect_tx(fb, (uint32_t)STAGE_BYTES);
                const size_t ta = ((size_t)tm * p.nkb + q) * OZ_A_BYTES, tb = ((size_t)tn * p.nkb + q) * OZ_B_BYTES;
#pragma unroll
                for (int i = 0; i < S; ++i) bulk_load(st + (uint32_t)(i * OZ_A_BYTES), p.a[i] + ta, OZ_A_BYTES, fb);
#pragma unroll
                for (int j = 0; j < S; ++j)
                    bulk_load(st + (uint32_t)(S * OZ_A_BYTES + j * OZ_B_BYTES), p.b[j] + tb, OZ_B_BYTES, fb);
                s_issued = gq + 1;
            }
        }
    } else if (warp == OZ_WARP_MMA && lane == 0) {
        // ---------------- MMA issuer: the S (S + 1) / 2 slice pairs of levels 0 .. S-1 as S products ----------------
        const uint64_t desc0 = sdesc_kmajor(smem_u32(smem), OZ_ROW);
        int gq = 0, gg = 0;  // k-blocks and k-block groups of this CTA so far
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        for (int q = 0; q < nk; ++q, ++gq) {
            const int s = gq % STAGES;
            const int g = gg + q / OZ_GROUP, a = g & 1;  // TMEM buffer a holds k-block group g
            const bool first = q % OZ_GROUP == 0, last = q % OZ_GROUP == OZ_GROUP - 1 || q == nk - 1;
            if (!mbar_wait(bar_full + 8 * s, (uint32_t)((gq / STAGES) & 1), abort_flag, p.err) ||
                (first && g >= 2 &&
                 !mbar_wait(bar_acc_empty + 8 * a, (uint32_t)(((g >> 1) - 1) & 1), abort_flag, p.err))) {
                stop = true;
                break;
            }
            tc_fence_after();
            const uint64_t dA = desc0 + (uint64_t)(s * (STAGE_BYTES >> 4));
            const uint64_t dB = dA + (uint64_t)(S * (OZ_A_BYTES >> 4));
            const uint32_t d = tmem + (uint32_t)(a * S * OZ_BN);
#pragma unroll
            for (int kk = 0; kk < OZ_ROW / 32; ++kk) {  // 16 BF16 values (32 bytes) of K per product
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    // A slice i times P slices 0 .. S-1-i into level blocks i .. S-1; the
                    // first product of a group (i = 0, all level blocks) overwrites them
                    mma_bf16(d + (uint32_t)(i * OZ_BN), dA + (uint64_t)(i * (OZ_A_BYTES >> 4) + 2 * kk),
                             dB + (uint64_t)(2 * kk), idesc_bf16(OZ_BM, OZ_BN * (S - i)),
                             (i > 0 || kk > 0 || !first) ? 1u : 0u);
                }
            }
            mma_commit(bar_empty + 8 * s);                // the stage may be refilled once these products finish
            if (last) mma_commit(bar_acc_full + 8 * a);  // the group's level sums are ready
            s_consumed = gq + 1;
        }
        gg += ng;
        }
        mma_commit(bar_done);
    } else if (warp < OZ_DRAIN_WARPS) {
        // ---------------- drain: exact integer level sums, then the FP64 epilogue ----------------
        const int quarter = warp & 3, cq = warp >> 2;  // TMEM lanes 32 quarter.., columns OZ_DC cq..
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cq * OZ_DC);
        int gg = 0;  // k-block groups drained by this CTA so far
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int tm, tn;
            tile_coords(t, p.tiles_m, p.tiles_n, 8, tm, tn);
            int acc[S][OZ_DC];
#pragma unroll
            for (int l = 0; l < S; ++l)
#pragma unroll
                for (int c = 0; c < OZ_DC; ++c) acc[l][c] = 0;
            for (int q = 0; q < ng; ++q, ++gg) {
                const int a = gg & 1;
                if (!mbar_wait(bar_acc_full + 8 * a, (uint32_t)((gg >> 1) & 1), abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // two levels per TMEM load round trip
#pragma unroll
                for (int l = 0; l < S; l += 2) {
                    uint32_t r[16];
                    tmem_ld8(lane_base + (uint32_t)((a * S + l) * OZ_BN), *reinterpret_cast<uint32_t(*)[8]>(r));
                    if (l + 1 < S)
                        tmem_ld8(lane_base + (uint32_t)((a * S + l + 1) * OZ_BN),
                                 *reinterpret_cast<uint32_t(*)[8]>(r + 8));
                    tmem_wait16(r);
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (l + h < S)
#pragma unroll
                            for (int c = 0; c < OZ_DC; ++c)
                                acc[l + h][c] += __float2int_rn(__uint_as_float(r[8 * h + c]));  // exact integers
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_acc_empty + 8 * a);
            }
            // the tile's FP64 results and epilogue; meanwhile the MMA warp fills the
            // freed TMEM buffers with the next tile's first groups
            const int grow = tm * OZ_BM + quarter * 32 + lane;  // row of the stacked batch entries
            if (ok && !*abort_flag && grow < p.nbatch * p.M) {
                const int b = grow / p.M, mm = grow - b * p.M;
                const int mh = mm / p.n, ml = mm - mh * p.n;
                const int code = p.rexp[grow];
                const bool nan_out = code == OZ_EXP_NONFINITE;
                // 2^(e_r - 8S) 2^(e_P - 8S + 1) 2^(8 (S - 1)) (sum_l S_l 2^(8 (S - 1 - l)))
                const int E = (code == OZ_EXP_ZERO || nan_out ? 0 : code) + p.p_exp - (2 * oz_frac(S) - 1) +
                              (S - 1) * OZ_BITS;
                const double scale = pow2(E);
#pragma unroll
                for (int c = 0; c < OZ_DC; ++c) {
                    const int nn = tn * OZ_BN + cq * OZ_DC + c;
                    if (nn >= p.n) continue;
                    double v;
                    if constexpr (S == 6) {
                        // levels in pairs 8 bits apart, then J = H_0 2^16 + H_1: all exact in int64
                        const long long H0 = (long long)acc[0][c] * 256 + acc[1][c];
                        const long long H1 = (long long)acc[2][c] * 256 + acc[3][c];
                        const long long H2 = (long long)acc[4][c] * 256 + acc[5][c];
                        v = oz_form6(H0 * 65536 + H1, H2, E, scale);
                    } else if constexpr (S == 5) {
                        // J = (S_0 2^8 + S_1) 2^16 + S_2 2^8 + S_3 (exact in int64), then + S_4
                        const long long H0 = (long long)acc[0][c] * 256 + acc[1][c];
                        const long long H1 = (long long)acc[2][c] * 256 + acc[3][c];
                        const long long J = H0 * 65536 + H1;
                        v = fma((double)J, pow2(OZ_BITS), (double)acc[4][c]) * scale;
                    } else {
                        // T = (S_0 2^8 + S_1) 2^16 + S_2 2^8 + S_3: exact in int64 (< 2^56), one rounding
                        const long long H0 = (long long)acc[0][c] * 256 + acc[1][c];
                        const long long H1 = (long long)acc[2][c] * 256 + acc[3][c];
                        v = (double)(H0 * 65536 + H1) * scale;
                    }
                    if (nan_out) v = __longlong_as_double(0x7ff8000000000000ll);
                    p.e.apply(b, mh, ml, nn, v);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == OZ_WARP_TMA && lane == 0) {
        if (*abort_flag) {
            // copies still in flight after an abort: wait for them (bounded) before exit
            for (int q = s_consumed; q < s_issued; ++q) {
                const int s = q % STAGES;
                const unsigned long long t0 = globaltimer();
                while (!mbar_try(bar_full + 8 * s, (uint32_t)((q / STAGES) & 1)) &&
                       globaltimer() - t0 < 100000000ull) {
                }
            }
        }
        const unsigned long long t0 = globaltimer();  // every product has completed
        while (!mbar_try(bar_done, 0u) && globaltimer() - t0 < 200000000ull) {
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == OZ_WARP_TMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

size_t oz_plane_bytes(long long rows, int n, int tile_rows) {
    return (size_t)((rows + tile_rows - 1) / tile_rows) * (size_t)((n + OZ_KV - 1) / OZ_KV) * (size_t)tile_rows * OZ_ROW;
}

cudaError_t oz_prepare() {
    static bool attr_set = false;
    if (attr_set) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute((const void*)ozaki_pass_kernel<6>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, oz_smem(6));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)ozaki_pass_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 oz_smem(5));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)ozaki_pass_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 oz_smem(4));
    attr_set = e == cudaSuccess;
    return e;
}

int oz_pairs(int s) { return s * (s + 1) / 2; }

// P's S slices below its scale 2^e_P > max |P| (returned): each value rounded once
// to t = round(p 2^(8S - 1 - e_P)), |t| <= 2^(8S - 1), and cut into S balanced
// base-256 digits (the last one |p_0| <= 128), as BF16 bit patterns (exact:
// integers of at most 8 significant bits), in tiled planes of 32-row tiles
// (oz_plane_bytes(n, n, 32) bytes each, cleared by the caller).
int oz_slice_host(const double* P, int n, int S, uint16_t* const planes[OZ_S]) {
    double pmax = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) pmax = fabs(P[i]) > pmax ? fabs(P[i]) : pmax;
    int ep = 0;
    frexp(pmax, &ep);
    const int nkb = (n + OZ_KV - 1) / OZ_KV;
    for (int r = 0; r < n; ++r)
        for (int k = 0; k < n; ++k) {
            long long t = llrint(ldexp(P[(size_t)r * n + k], oz_frac(S) - 1 - ep));
            float dig[OZ_S];
            for (int i = S - 1; i > 0; --i) {
                const long long d = ((t + 128) & 255) - 128;
                dig[i] = (float)d;
                t = (t - d) / 256;  // exact: t - d is a multiple of 256
            }
            dig[0] = (float)t;
            const long long o = oz_tile_off(r, k, nkb, 5);
            for (int i = 0; i < S; ++i) {
                uint32_t bits;
                memcpy(&bits, &dig[i], 4);
                planes[i][o] = (uint16_t)(bits >> 16);  // exact: at most 8 significant bits
            }
        }
    return ep;
}

namespace {

template <int S>
cudaError_t launch_ozaki_pass_s(void* const pslices[OZ_S], int p_exp, const double* A, int M, int n, int nbatch,
                                int ld, void* const slices[OZ_S], int* rexp, const Epi<double>& e, unsigned* err,
                                cudaStream_t st) {
    OzPlanes planes;
    for (int i = 0; i < OZ_S; ++i) planes.s[i] = static_cast<__nv_bfloat16*>(slices[i]);
    const long long rows = (long long)nbatch * M;
    const int nkb = (n + OZ_KV - 1) / OZ_KV;
    if (n >= OZ_SLICE_ROW_MIN) {
        if (n > OZ_MAX_N || rows > 0x7FFFFFFFll) return cudaErrorInvalidValue;  // one block per row, at most 1024 threads
        oz_slice_row_kernel<S><<<(unsigned)rows, oz_slice_row_threads(n), 0, st>>>(A, n, ld, nkb, rexp, planes);
    } else {
        long long blocks = (rows + 7) / 8;  // one warp per row
        if (blocks > 152 * 16) blocks = 152 * 16;
        oz_slice_kernel<S><<<(unsigned)blocks, 256, 0, st>>>(A, rows, n, ld, nkb, rexp, planes);
    }
    OzParams p;
    for (int i = 0; i < OZ_S; ++i) {
        p.a[i] = static_cast<const uint8_t*>(slices[i]);
        p.b[i] = static_cast<const uint8_t*>(pslices[i]);
    }
    p.nkb = nkb;
    p.M = M;
    p.n = n;
    p.nbatch = nbatch;
    p.p_exp = p_exp;
    p.tiles_m = (int)((rows + OZ_BM - 1) / OZ_BM);
    p.tiles_n = (n + OZ_BN - 1) / OZ_BN;
    p.rexp = rexp;
    p.err = err;
    p.e = e;
    // persistent: one CTA per SM walks the tiles (grid = min(tiles, SMs))
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    }
    const long long ntiles = (long long)p.tiles_m * p.tiles_n;
    ozaki_pass_kernel<S><<<(unsigned)(ntiles < sms ? ntiles : sms), OZ_THREADS, oz_smem(S), st>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ozaki_pass(int S, void* const pslices[OZ_S], int p_exp, const double* A, int M, int n,
                              int nbatch, int ld, void* const slices[OZ_S], int* rexp, const Epi<double>& e,
                              unsigned* err, cudaStream_t st) {
    if (S == 6) return launch_ozaki_pass_s<6>(pslices, p_exp, A, M, n, nbatch, ld, slices, rexp, e, err, st);
    if (S == 5) return launch_ozaki_pass_s<5>(pslices, p_exp, A, M, n, nbatch, ld, slices, rexp, e, err, st);
    if (S == 4) return launch_ozaki_pass_s<4>(pslices, p_exp, A, M, n, nbatch, ld, slices, rexp, e, err, st);
    return cudaErrorInvalidValue;
}

}  // namespace etd
