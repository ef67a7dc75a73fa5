// Internal declarations of the ETD2RK-DS CUDA library (not part of the C ABI).
//
// Data layout of every internal field buffer: [comp][slow][mid][fast] with the
// fast axis padded to `ld` elements (a multiple of 4 so that every row starts on
// a 16-byte boundary, as TMA requires). One transform pass is the product
//     out(b, mm, nn) = sum_k A[b][mm][k] * P[nn][k]
// over the fast axis k of A (rows mm = the n^(d-1) other indices), written
// TRANSPOSED so that the contracted axis becomes the slowest one:
//     out offset = (nn * n^(d-2) + mm / n) * ld + mm % n.
// P is the symmetric orthogonal sine basis, so two passes give P X P (2D) and
// three passes the three mode products (3D), and the same passes invert them.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/etd.h"

namespace etd {

enum EpiMode : int {
    EPI_SPLIT = 0,   // write the value as the next pass's operand
    EPI_CARRY = 1,   // store the carried spectral state  U^ = value
    EPI_STAGE1 = 2,  // eq. (13) in the spectral basis -> W^, F^q, operand(W^)
    EPI_STAGE2 = 3,  // eq. (14) in the spectral basis -> U^+, operand(U^+)
    EPI_PLAIN = 4,   // store the physical field (rows of length n, own pitch)
    // Reaction fused into the epilogue (reactions that act on each component at a
    // point on its own, rx_fusable): the value is a physical field value w, and
    EPI_REACT = 5,       // f(w) is written as the next pass's operand (step a5 from a4)
    EPI_PLAIN_REACT = 6  // w is stored as EPI_PLAIN does, and f(w) as the operand (a1 of the
                         // next step from a7)
};

// Reactions the epilogue can evaluate: f at a point depends only on the same
// component's value there (f = 0, c u, u - u^3, rho u / (1 - u)), so the thread
// that holds one output value has all it needs. FitzHugh-Nagumo couples the two
// components (held by different CTAs) and the manufactured forcing needs FP64
// coordinates: those keep the reaction kernel.
__host__ __device__ __forceinline__ bool rx_fusable(int kind) {
    return kind == ETD_RX_NONE || kind == ETD_RX_LINEAR || kind == ETD_RX_ALLEN_CAHN || kind == ETD_RX_SINGULAR;
}

// f(w) of a fusable reaction, in the arithmetic of the reaction kernel.
template <typename T>
__device__ __forceinline__ T rx_point(int kind, T c, T w) {
    switch (kind) {
        case ETD_RX_LINEAR:
            return c * w;
        case ETD_RX_ALLEN_CAHN:
            return w - w * w * w;
        case ETD_RX_SINGULAR:
            return c * w / ((T)1 - w);
        default:
            return (T)0;
    }
}

// How an operand is written for the tensor-core products.
enum SplitKind : int {
    SPLIT_NONE = 0,     // one plane, the value itself (CUDA-core products)
    SPLIT_TF32 = 1,     // hi = rna_tf32(v), lo = rna_tf32(v - hi)
    SPLIT_TF32_HI = 2,  // hi only, rna_tf32(v) (single TF32 product)
    SPLIT_TF32_3 = 3,   // hi, mid = rna_tf32(v - hi), lo = rna_tf32(v - hi - mid)
    SPLIT_BF16_2 = 4,   // BF16 planes: hi = rn_bf16(v), lo = rn_bf16(v - hi)
    SPLIT_BF16_3 = 5    // BF16 planes: hi, mid, lo (24 significant bits)
};

// BF16 pieces of an FP32 value in FP32 arithmetic: each residual v - piece is
// exact in FP32 (the piece keeps fewer bits than v), so no FP64 is needed.
__device__ __forceinline__ void split_bf16_f(float v, int pieces, __nv_bfloat16* hi, __nv_bfloat16* lo,
                                             __nv_bfloat16* lo2, long long o) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[o] = h;
    if (pieces < 2) return;
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    lo[o] = m;
    if (pieces < 3) return;
    lo2[o] = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

enum ErrBits : unsigned { ERR_TIMEOUT = 1u, ERR_BAD_CONFIG = 2u, ERR_DIVERGED = 4u };

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Two floats that hold BF16 values exactly, packed as a bfloat162 word (a low).
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// ---- double-float arithmetic ----
// A double-float is the unevaluated sum x + y of two floats with |y| <= ulp(x)/2,
// about 48 significant bits. GB300 runs FP64 at a small fraction of its FP32
// rate, so the per-element updates of the carried spectral state in the FP32
// paths use these error-free transformations in FP32: Knuth's TwoSum and the
// FMA form of Dekker's TwoProduct. The _rn intrinsics keep the compiler from
// contracting a product and a sum into one FMA, which would break exactness.
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {  // a + b exactly
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);  // exact rounding error of p
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    float e = __fmaf_rn(a.x, b, -p);
    e = __fmaf_rn(a.y, b, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float2 s = ff_two_sum(a.x, b.x);
    return ff_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 ff_add_f(float2 a, float b) {  // a + b for a float b
    const float2 s = ff_two_sum(a.x, b);
    return ff_fast_two_sum(s.x, __fadd_rn(s.y, a.y));
}

// Operand pieces of a double-float w: piece 0 rounds w.x, piece j rounds what
// the earlier pieces left of w.x + w.y. Each w.x - piece0 is exact in FP32.
template <bool BF16>
__device__ __forceinline__ float piece_round(float v) {
    if constexpr (BF16) return __bfloat162float(__float2bfloat16_rn(v));
    else return tf32_rna(v);
}
template <bool BF16>
__device__ __forceinline__ void ff_pieces(float2 w, float* q) {
    q[0] = piece_round<BF16>(w.x);
    const float r1 = __fsub_rn(w.x, q[0]);
    q[1] = piece_round<BF16>(__fadd_rn(r1, w.y));
    q[2] = piece_round<BF16>(__fadd_rn(__fsub_rn(r1, q[1]), w.y));
}

// The carried spectral state and the factor grids carry more than FP32
// precision for every precision: in the eigenbasis the linear part of a step is
// the elementwise product E1x E1y.. U^, so rounding the state or the factors to
// FP32 would add a systematic relative error of up to 2^-24 per step (about
// N 2^-24 after N steps). The FP64 path holds them in FP64 (St = double); the
// FP32 paths hold double-floats (St = float2, same 8 bytes per value) and update
// them in FP32 arithmetic. Only the transform operands and the physical fields use T.
//
// The two Hadamard stages of a step (eq. (13)-(14) in the eigenbasis, with
// S = E_1(tau A_2) [E_1(tau A_2^z)] at the y [z] modes and E_l at the x mode):
//   stage 1, value F^ = T f(U):   W^ = S (E1 U^ + tau E2 F^),  Z = W^ - tau E3 S F^
//   stage 2, value F_W^ = T f(W): U^+ = Z + tau E3 F_W^
// Z is eq. (14)'s W^ + tau E3 (F_W^ - S F^) with its F_W^-free part formed in
// stage 1, so stage 2 reads one state value per point instead of W^ and S F^.
template <typename T>
struct Epi {
    using St = typename std::conditional<sizeof(T) == 4, float2, double>::type;
    int mode;        // EpiMode
    int split;       // SplitKind (float only)
    int d, n, M;     // M = n^(d-1) rows per component
    int mq;          // M / n = n^(d-2)
    int ld;          // padded row length of internal buffers
    long long bs;    // component stride of internal buffers (elements)
    T* op_hi;        // operand output planes (layout of the next pass)
    T* op_lo;
    T* op_lo2;       // third piece (SPLIT_TF32_3)
    T* dst;          // EPI_PLAIN destination
    int ld_dst;
    long long bs_dst;
    St* uhat;        // carried spectral state U^   (internal layout)
    St* zhat;        // Z of the current step (stage 1 -> stage 2)
    const St* grid;  // [comp][3][n]: E_1, tau E_2, tau E_3 at tau * lambda_k
    int rx;          // EPI_REACT / EPI_PLAIN_REACT: the reaction (rx_fusable)
    T rx_c;          // its parameter (c of ETD_RX_LINEAR, rho of ETD_RX_SINGULAR)

    __device__ __forceinline__ void write_operand(long long o, double v) const {
        op_hi[o] = (T)v;  // FP64 path: one plane, CUDA-core products
    }

    // Operand pieces of an FP32 value, FP32 arithmetic only (split and reaction passes).
    __device__ __forceinline__ void write_operand_f(long long o, float v) const {
        if constexpr (sizeof(T) == 4) {
            write_operand_ff(o, make_float2(v, 0.f));
        } else {
            write_operand(o, (double)v);
        }
    }

    // Operand pieces of a double-float value (FP32 paths).
    __device__ __forceinline__ void write_operand_ff(long long o, float2 w) const {
        if constexpr (sizeof(T) == 4) {
            float q[3];
            if (split == SPLIT_BF16_2 || split == SPLIT_BF16_3) {
                ff_pieces<true>(w, q);
                __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(op_hi);
                h[o] = __float2bfloat16_rn(q[0]);  // exact: q[0] is a BF16 value
                reinterpret_cast<__nv_bfloat16*>(op_lo)[o] = __float2bfloat16_rn(q[1]);
                if (split == SPLIT_BF16_3) reinterpret_cast<__nv_bfloat16*>(op_lo2)[o] = __float2bfloat16_rn(q[2]);
                return;
            }
            if (split == SPLIT_TF32 || split == SPLIT_TF32_3) {
                ff_pieces<false>(w, q);
                op_hi[o] = q[0];
                op_lo[o] = q[1];
                if (split == SPLIT_TF32_3) op_lo2[o] = q[2];
                return;
            }
            if (split == SPLIT_TF32_HI) {
                op_hi[o] = tf32_rna(w.x);
                return;
            }
            op_hi[o] = __fadd_rn(w.x, w.y);
        }
    }

    // Does this epilogue read carried state (U^ in stage 1, Z in stage 2)?
    __device__ __forceinline__ bool reads_state() const { return mode == EPI_STAGE1 || mode == EPI_STAGE2; }
    __device__ __forceinline__ const St* state_in() const { return mode == EPI_STAGE1 ? uhat : zhat; }

    // Value v = out(b, mm, nn) with mm = mh * n + ml.
    __device__ __forceinline__ void apply(int b, int mh, int ml, int nn, T v) const;
};

// State values of up to N consecutive columns nn0 .. nn0+count-1 of one row
// (mm = mh * n + ml) for the epilogue below. Callers issue this for the next
// batch of columns before they apply the current one, so the loads overlap the
// arithmetic and stores of the current batch.
template <int N>
__device__ __forceinline__ void epi_load_state(const Epi<float>& e, int b, int mh, int ml, int nn0, int count,
                                               float2 (&st)[N]) {
    if (!e.reads_state()) return;
    const float2* src = e.state_in() + (long long)b * e.bs + ((long long)nn0 * e.mq + mh) * e.ld + ml;
    const long long step = (long long)e.mq * e.ld;  // offset between consecutive nn
#pragma unroll
    for (int j = 0; j < N; ++j) st[j] = (j < count) ? src[j * step] : make_float2(0.f, 0.f);
}

// Epilogue of up to N consecutive columns of one row, values v[], state st[]
// from epi_load_state (FP32 paths).
template <int N>
__device__ __forceinline__ void epi_apply_batch(const Epi<float>& e, int b, int mh, int ml, int nn0, const float* v,
                                                int count, const float2 (&st)[N]) {
    const long long base = (long long)b * e.bs + (long long)mh * e.ld + ml;
    const long long step = (long long)e.mq * e.ld;  // offset between consecutive nn
    if (e.mode == EPI_PLAIN || e.mode == EPI_PLAIN_REACT) {
        float* d = e.dst + (long long)b * e.bs_dst + ((long long)nn0 * e.mq + mh) * e.ld_dst + ml;
        const long long sd = (long long)e.mq * e.ld_dst;
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j < count) d[j * sd] = v[j];
        if (e.mode == EPI_PLAIN) return;
    }
    const long long o0 = base + (long long)nn0 * step;
    if (e.mode == EPI_SPLIT) {
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j < count) e.write_operand_f(o0 + j * step, v[j]);
        return;
    }
    if (e.mode == EPI_REACT || e.mode == EPI_PLAIN_REACT) {  // f(w) as the next pass's operand
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j < count) e.write_operand_f(o0 + j * step, rx_point<float>(e.rx, e.rx_c, v[j]));
        return;
    }
    if (e.mode == EPI_CARRY) {
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j < count) e.uhat[o0 + j * step] = make_float2(v[j], 0.f);
        return;
    }
    // The transformed reaction v carries the transform's relative error (about
    // 2^-22 for split TF32), so its products with S, tau E2 and tau E3 are formed
    // in FP32 (relative error about 2^-23) and added to the double-float term
    // S E1 U^, which keeps double-float precision and is formed once for both W^
    // and Z.
    const float2* g = e.grid + (long long)b * 3 * e.n;
    const float g3 = g[2 * e.n + ml].x;
    if (e.mode == EPI_STAGE1) {
        // W^ = S (E1 U^ + tau E2 F^),  Z = W^ - tau E3 S F^ = S (E1 U^ + (tau E2 - tau E3) F^)
        const float2 g1 = g[ml], g2 = g[e.n + ml];
        const float g23 = __fsub_rn(g2.x, g3) + g2.y - g[2 * e.n + ml].y;
        const float2 gm = g[mh];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j < count) {
                const long long o = o0 + j * step;
                const float2 sl = g[nn0 + j];
                const float2 sj = (e.d == 2) ? sl : ff_mul(gm, sl);
                const float2 su = ff_mul(ff_mul(g1, st[j]), sj);  // S E1 U^, double-float
                const float sv = __fmul_rn(sj.x, v[j]);              // S F^, FP32
                const float2 w = ff_add_f(su, __fmul_rn(g2.x, sv));
                e.zhat[o] = ff_add_f(su, __fmul_rn(g23, sv));
                e.write_operand_ff(o, w);
            }
        }
        return;
    }
    if (e.mode == EPI_STAGE2) {  // U^+ = Z + tau E3 F_W^
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j < count) {
                const long long o = o0 + j * step;
                const float2 u = ff_add_f(st[j], __fmul_rn(g3, v[j]));
                e.uhat[o] = u;
                e.write_operand_ff(o, u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Row-vector epilogue (FP32 paths): eight consecutive rows ml0 .. ml0+7 of one
// (component, mh) and one column nn, so every store and state load of the
// batch is a 16-byte access along the contiguous ml direction instead of eight
// 2- to 8-byte accesses at the column stride. The per-element arithmetic is the
// same as in epi_apply_batch (results are bitwise identical). Valid only when
// epi_rows8_ok() holds on the host (n, pitches and strides multiples of 8,
// 16-byte aligned planes); ml0 is then a multiple of 8.
__host__ __device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

inline bool epi_rows8_ok(const Epi<float>& e) {
    if (e.n % 8 != 0 || e.ld % 8 != 0 || e.bs % 8 != 0) return false;
    if (!aligned16(e.op_hi) || !aligned16(e.op_lo) || !aligned16(e.op_lo2)) return false;
    if (!aligned16(e.uhat) || !aligned16(e.zhat) || !aligned16(e.grid)) return false;
    if ((e.mode == EPI_PLAIN || e.mode == EPI_PLAIN_REACT) &&
        (e.ld_dst % 8 != 0 || e.bs_dst % 8 != 0 || !aligned16(e.dst)))
        return false;
    return true;
}

__device__ __forceinline__ void epi_load_rows8(const Epi<float>& e, int b, int mh, int ml0, int nn, float4 (&st)[4]) {
    if (!e.reads_state()) return;
    const float4* src = reinterpret_cast<const float4*>(e.state_in() + (long long)b * e.bs +
                                                        ((long long)nn * e.mq + mh) * e.ld + ml0);
#pragma unroll
    for (int i = 0; i < 4; ++i) st[i] = __ldg(src + i);  // state_in is never written by the same pass
}

__device__ __forceinline__ void store8(float* d, const float (&x)[8]) {
    reinterpret_cast<float4*>(d)[0] = make_float4(x[0], x[1], x[2], x[3]);
    reinterpret_cast<float4*>(d)[1] = make_float4(x[4], x[5], x[6], x[7]);
}

__device__ __forceinline__ void store8_ff(float2* d, const float2 (&w)[8]) {
    float4* q = reinterpret_cast<float4*>(d);
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = make_float4(w[2 * i].x, w[2 * i].y, w[2 * i + 1].x, w[2 * i + 1].y);
}

// Operand pieces of eight double-float values at o .. o+7 (write_operand_ff per
// element), packed as they are formed: one 16-byte store per BF16 piece plane,
// two per TF32 plane.
__device__ __forceinline__ void write_operand_ff8(const Epi<float>& e, long long o, const float2 (&w)[8]) {
    if (e.split == SPLIT_BF16_2 || e.split == SPLIT_BF16_3) {
        uint32_t h[4], l[4], l2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float a[3], b[3];
            ff_pieces<true>(w[2 * k], a);
            ff_pieces<true>(w[2 * k + 1], b);
            h[k] = bf16x2_bits(a[0], b[0]);
            l[k] = bf16x2_bits(a[1], b[1]);
            l2[k] = bf16x2_bits(a[2], b[2]);
        }
        *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(e.op_hi) + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(e.op_lo) + o) = make_uint4(l[0], l[1], l[2], l[3]);
        if (e.split == SPLIT_BF16_3)
            *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(e.op_lo2) + o) =
                make_uint4(l2[0], l2[1], l2[2], l2[3]);
        return;
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {  // four values per 16-byte store
        float q0[4], q1[4], q2[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 x = w[4 * g + i];
            if (e.split == SPLIT_TF32 || e.split == SPLIT_TF32_3) {
                float q[3];
                ff_pieces<false>(x, q);
                q0[i] = q[0];
                q1[i] = q[1];
                q2[i] = q[2];
            } else {
                q0[i] = (e.split == SPLIT_TF32_HI) ? tf32_rna(x.x) : __fadd_rn(x.x, x.y);
                q1[i] = q2[i] = 0.f;
            }
        }
        reinterpret_cast<float4*>(e.op_hi + o)[g] = make_float4(q0[0], q0[1], q0[2], q0[3]);
        if (e.split == SPLIT_TF32 || e.split == SPLIT_TF32_3)
            reinterpret_cast<float4*>(e.op_lo + o)[g] = make_float4(q1[0], q1[1], q1[2], q1[3]);
        if (e.split == SPLIT_TF32_3) reinterpret_cast<float4*>(e.op_lo2 + o)[g] = make_float4(q2[0], q2[1], q2[2], q2[3]);
    }
}

__device__ __forceinline__ void epi_apply_rows8(const Epi<float>& e, int b, int mh, int ml0, int nn, const float (&v)[8],
                                                const float4 (&st4)[4]) {
    if (e.mode == EPI_PLAIN || e.mode == EPI_PLAIN_REACT) {
        store8(e.dst + (long long)b * e.bs_dst + ((long long)nn * e.mq + mh) * e.ld_dst + ml0, v);
        if (e.mode == EPI_PLAIN) return;
    }
    const long long o = (long long)b * e.bs + ((long long)nn * e.mq + mh) * e.ld + ml0;
    float2 w[8];
    if (e.mode == EPI_REACT || e.mode == EPI_PLAIN_REACT) {  // f(w) as the next pass's operand
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = make_float2(rx_point<float>(e.rx, e.rx_c, v[i]), 0.f);
        write_operand_ff8(e, o, w);
        return;
    }
    if (e.mode == EPI_SPLIT || e.mode == EPI_CARRY) {
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = make_float2(v[i], 0.f);
        if (e.mode == EPI_SPLIT)
            write_operand_ff8(e, o, w);
        else
            store8_ff(e.uhat + o, w);
        return;
    }
    float2 st[8];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        st[2 * i] = make_float2(st4[i].x, st4[i].y);
        st[2 * i + 1] = make_float2(st4[i].z, st4[i].w);
    }
    const float2* g = e.grid + (long long)b * 3 * e.n;
    if (e.mode == EPI_STAGE1) {
        const float2 sl = g[nn];
        const float2 sj = (e.d == 2) ? sl : ff_mul(g[mh], sl);
        float4* zq = reinterpret_cast<float4*>(e.zhat + o);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 z[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = 2 * k + h, ml = ml0 + i;
                const float2 g1 = g[ml], g2 = g[e.n + ml], g3v = g[2 * e.n + ml];
                const float g23 = __fsub_rn(g2.x, g3v.x) + g2.y - g3v.y;
                const float2 su = ff_mul(ff_mul(g1, st[i]), sj);  // S E1 U^, double-float
                const float sv = __fmul_rn(sj.x, v[i]);              // S F^, FP32
                w[i] = ff_add_f(su, __fmul_rn(g2.x, sv));
                z[h] = ff_add_f(su, __fmul_rn(g23, sv));
            }
            zq[k] = make_float4(z[0].x, z[0].y, z[1].x, z[1].y);
        }
        write_operand_ff8(e, o, w);
        return;
    }
    if (e.mode == EPI_STAGE2) {  // U^+ = Z + tau E3 F_W^
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = ff_add_f(st[i], __fmul_rn(g[2 * e.n + ml0 + i].x, v[i]));
        store8_ff(e.uhat + o, w);
        write_operand_ff8(e, o, w);
    }
}

template <typename T>
__device__ __forceinline__ void Epi<T>::apply(int b, int mh, int ml, int nn, T v) const {
    if constexpr (sizeof(T) == 4) {
        float2 st[1];
        epi_load_state<1>(*this, b, mh, ml, nn, 1, st);
        epi_apply_batch<1>(*this, b, mh, ml, nn, &v, 1, st);
    } else {
        if (mode == EPI_PLAIN || mode == EPI_PLAIN_REACT) {
            dst[b * bs_dst + ((long long)nn * mq + mh) * ld_dst + ml] = v;
            if (mode == EPI_PLAIN) return;
        }
        const long long o = b * bs + ((long long)nn * mq + mh) * ld + ml;
        if (mode == EPI_REACT || mode == EPI_PLAIN_REACT) {
            write_operand(o, rx_point<double>(rx, rx_c, v));
            return;
        }
        const double* g = grid + (long long)b * 3 * n;
        switch (mode) {
            case EPI_SPLIT:
                write_operand(o, v);
                break;
            case EPI_CARRY:
                uhat[o] = v;
                break;
            case EPI_STAGE1: {
                // spectral indices: k = ml (x mode); 2D l = nn; 3D l = mh, p = nn
                const double s = (d == 2) ? g[nn] : g[mh] * g[nn];  // E_1(tau A_2) [E_1(tau A_2^z)]
                const double w = (g[ml] * uhat[o] + g[n + ml] * v) * s;
                zhat[o] = w - g[2 * n + ml] * (s * v);
                write_operand(o, w);
                break;
            }
            case EPI_STAGE2: {
                const double u = zhat[o] + g[2 * n + ml] * v;
                uhat[o] = u;
                write_operand(o, u);
                break;
            }
            default:
                break;
        }
    }
}

// Reaction / split kernel arguments (steps a1 and a5).
template <typename T>
struct Rx {
    int kind;        // ETD_RX_*, or -1 for "identity" (split u itself)
    int ncomp, n;
    int ninst;       // instances; instance i's component c starts at (i * ncomp + c) * bs
    long long npts;  // n^d
    const T* in;
    int ld_in;
    long long bs_in;
    T* out_hi;
    T* out_lo;
    T* out_lo2;
    int ld_out;
    long long bs_out;
    int split;
    T rp[4];
    // ETD_RX_AC_FORCED: psi(x, t) = (-lambda + d pi^2 kappa) e u0 - e u0 (1 - (e u0)^2), e = e^{-lambda t}
    int d;
    double decay;     // e^{-lambda t}
    double psi_coef;  // -lambda + d pi^2 kappa
};

// Record the message etd_last_error() returns on this host thread (etd_plan.cu).
void set_last_error(const char* msg);

// ---- adjoint step (adjoint.cu) ----
// out = alpha * Xa * [S] * in1 + beta * Xb * [S] * in2 over the spectral grid,
// X* selected from {1, E1, tau E2, tau E3} at the x mode, S = E1 at the other modes.
template <typename T>
struct SpecCombine {
    int ncomp, d, n;
    long long npts;
    const double* grid;
    const float2* grid2;  // double-float copy (FP32 paths)
    const T* in1;
    int xsel1, s1;
    double alpha;
    const T* in2;
    int xsel2, s2;
    double beta;
    T* out;
};
template <typename T>
struct ReactVjp {  // out = base + J_f(X)^T V
    int kind, ncomp;
    long long npts;
    double rp[4];
    const T* X;
    const T* V;
    const T* base;
    T* out;
};
template <typename T>
struct GradKappa {
    int ncomp, d, n;
    long long npts;
    const double* grid;
    const double* dgrid;  // kappa derivatives of E1, tau E2, tau E3
    const float2* grid2;  // double-float copies (FP32 paths)
    const float2* dgrid2;
    const T* Lh;          // U+bar^
    const T* Gbh;         // Gbar^
    const T* Wbh;         // Wbar^
    const T* Uh;          // U^
    const T* Fh;          // F^
    const T* FWh;         // F_W^
    double* out;          // [ncomp], accumulated
};
template <typename T>
struct GradRx {
    int kind, ncomp;
    long long npts;
    double rp[4];
    const T* U;
    const T* W;
    const T* Gb;
    const T* Fb;
    double* out;  // [4], accumulated
};
template <typename T>
void launch_spec_combine(const SpecCombine<T>& a, cudaStream_t st);
template <typename T>
void launch_react_vjp(const ReactVjp<T>& a, cudaStream_t st);
template <typename T>
void launch_grad_kappa(const GradKappa<T>& a, cudaStream_t st);
template <typename T>
void launch_grad_rx(const GradRx<T>& a, cudaStream_t st);

// ---- launchers (defined in the .cu files) ----
void launch_gemm_simt_f32(const float* A, const float* P, int M, int n, int nbatch, const Epi<float>& e,
                          cudaStream_t st);
void launch_gemm_simt_f64(const double* A, const double* P, int M, int n, int nbatch, const Epi<double>& e,
                          cudaStream_t st);
void launch_react_f32(const Rx<float>& r, cudaStream_t st);
// ETD_PREC_DST32: one transform pass as FFT-based DST-I of every row of A
// (n + 1 a power of two), through tmp (nbatch * M rows of pitch ld) and the epilogue.
cudaError_t launch_dst_pass(const float* A, int M, int n, int nbatch, int ld, long long bs, const float2* tw,
                            float* tmp, const Epi<float>& e, cudaStream_t st);
void launch_react_f64(const Rx<double>& r, cudaStream_t st);
void launch_stats_f32(const float* u, long long count, double* acc, cudaStream_t st);
// *flag |= 1 if the byte ranges a and b (16-byte aligned, length a multiple of 4) differ.
void launch_differ(const void* a, const void* b, size_t bytes, unsigned* flag, cudaStream_t st);
void launch_stats_f64(const double* u, long long count, double* acc, cudaStream_t st);
// In-step check (step a8): after launch_stats_* into acc[0..1], raise ERR_DIVERGED
// in err[0] when acc holds a non-finite count or max |u| > limit > 0; the first
// failure records its step in err[1] and max |u|, count in saved[0..1].
void launch_diag_check(const double* acc, double limit, unsigned step, unsigned* err, double* saved,
                       cudaStream_t st);

// tcgen05 transform pass (gemm_tc.cu)
struct TcConfig {
    int bn;          // tile width along nn (multiple of 32, <= 256)
    int stages;      // shared-memory pipeline depth
    int products;    // 1 (TF32), 3 (two-piece split) or 6 (three-piece split)
    int pieces;      // operand pieces read per product mode
    bool bf16;       // BF16 pieces, kind::f16 products (else TF32 pieces, kind::tf32)
    bool accurate;   // separate correction accumulator + compensated k-block sums
    bool persistent; // one CTA per SM, epilogue overlapped with the next tile
    int tiles_m, tiles_n;
    int tmem_cols;
    int smem_bytes;
    unsigned stage_bytes;
};
struct TcMaps;  // opaque holder of CUtensorMap objects (gemm_tc.cu)
// accurate: the ACCURATE variant (three pieces only): correction products in
// their own accumulator, compensated sums across k-blocks
TcConfig tc_choose(int M, int n, int products, int nbatch, bool bf16, bool accurate);
// The configurations an autotuner may time for one pass (the tc_choose rule's
// choice first, then the other kernel / tile widths that can run it); returns
// how many were written to out (at most max_out).
int tc_candidates(int M, int n, int products, int nbatch, bool bf16, bool accurate, TcConfig* out, int max_out);
// a[i][j]: operand buffer i, piece j (NULL = reuse piece 0); pp[j]: pieces of P;
// bn_slot: tile widths of the two configurations the maps serve.
cudaError_t tc_maps_create(TcMaps** out, int M, int n, int nbatch, int ld, const void* const a[][3], int n_a,
                           const void* const pp[3], const int bn_slot[2], bool bf16);
void tc_maps_destroy(TcMaps* m);
cudaError_t launch_gemm_tc(const TcConfig& cfg, int slot, const TcMaps* maps, int a_index, int M, int n, int nbatch,
                           const Epi<float>& e, unsigned* err, cudaStream_t st);
const char* tc_last_driver_error();

// ETD_PREC_FP64_SPLIT (6 slices), _SPLIT40 (5) and _SPLIT32 (4) transform pass
// (ozaki.cu): FP64 operands cut into balanced 8-bit digits (BF16 slices) below a
// per-row power-of-two scale, exact slice products on the tensor cores, FP64 result
// through the Epi<double> epilogue.
constexpr int OZ_S = 6;          // the most slices a precision uses (planes allocated per plan: its own count)
constexpr int OZ_MAX_N = 16384;  // K <= 16384 keeps the int32 level sums exact
int oz_pairs(int s);             // slice products per MMA tile and k-step: s (s + 1) / 2
constexpr int OZ_TILE_ROWS_A = 128;  // rows of an operand slice tile (the MMA's M)
constexpr int OZ_TILE_ROWS_P = 32;   // rows of a P slice tile (the output tile's width)
// Bytes of one tiled slice plane of `rows` rows of n values: tiles of tile_rows
// rows x 32 values, the rows and the last k-block padded (padding must be zero).
size_t oz_plane_bytes(long long rows, int n, int tile_rows);
// Once per process, before the first pass: the product kernel's shared-memory size.
cudaError_t oz_prepare();
// P's slices on the host (n x n, into tiled planes of OZ_TILE_ROWS_P-row tiles,
// zeroed by the caller); returns P's scale exponent e_P (max |P| < 2^e_P)
int oz_slice_host(const double* P, int n, int s, uint16_t* const planes[OZ_S]);
// The pass: A's row scales into rexp (nbatch * M ints) and its slices into the
// tiled planes `slices` (OZ_TILE_ROWS_A-row tiles), then the products with P's
// tiled slice planes `pslices` and the epilogue.
cudaError_t launch_ozaki_pass(int s, void* const pslices[OZ_S], int p_exp, const double* A, int M, int n,
                              int nbatch, int ld, void* const slices[OZ_S], int* rexp, const Epi<double>& e,
                              unsigned* err, cudaStream_t st);
cudaError_t launch_wait_timeout_probe(unsigned* err, double limit_ms, cudaStream_t st);

}  // namespace etd
