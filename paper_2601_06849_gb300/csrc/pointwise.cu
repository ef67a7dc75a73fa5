// Pointwise kernels of the ETD2RK-DS step:
//   - the reaction f(t, u) of all components at one grid point (steps a1 and
//     a5: f(t_n, U) in eq. (13), f(t_{n+1}, W) in eq. (14)), written straight
//     into the operand planes of the next transform pass;
//   - FP64 field diagnostics (step a8): max |u| and the count of non-finite values,
//     and the in-step check of those against the plan's bound.
// Both are bandwidth-bound: one read of each component and one write of each
// operand plane per point.
#include "etd_internal.cuh"
#include "../../include/etd.h"

namespace etd {

template <typename T>
__device__ __forceinline__ void store_split(T* hi, T* lo, T* lo2, long long o, T v, int split) {
    if constexpr (sizeof(T) == 4) {
        if (split == SPLIT_BF16_2 || split == SPLIT_BF16_3) {
            split_bf16_f(v, split == SPLIT_BF16_3 ? 3 : 2, reinterpret_cast<__nv_bfloat16*>(hi),
                         reinterpret_cast<__nv_bfloat16*>(lo), reinterpret_cast<__nv_bfloat16*>(lo2), o);
            return;
        }
        if (split == SPLIT_TF32_3) {  // three TF32 pieces hold all 24 bits of v
            const float h = tf32_rna(v);
            const float m = tf32_rna(v - h);
            hi[o] = h;
            lo[o] = m;
            lo2[o] = tf32_rna(v - h - m);
            return;
        }
        if (split == SPLIT_TF32) {
            float h = tf32_rna(v);
            hi[o] = h;
            lo[o] = tf32_rna(v - h);
            return;
        }
        if (split == SPLIT_TF32_HI) {
            hi[o] = tf32_rna(v);
            return;
        }
    }
    hi[o] = v;
}

// Operand pieces of two adjacent values (element index o even): one 4-byte
// (BF16 pair) or 8-byte (float pair) store per plane.
__device__ __forceinline__ void store_split2(float* hi, float* lo, float* lo2, long long o, float va, float vb,
                                             int split) {
    if (split == SPLIT_BF16_2 || split == SPLIT_BF16_3) {
        const __nv_bfloat16 ha = __float2bfloat16_rn(va), hb = __float2bfloat16_rn(vb);
        const float ra = va - __bfloat162float(ha), rb = vb - __bfloat162float(hb);  // exact
        const __nv_bfloat16 ma = __float2bfloat16_rn(ra), mb = __float2bfloat16_rn(rb);
        reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(hi) + o)[0] = __halves2bfloat162(ha, hb);
        reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(lo) + o)[0] = __halves2bfloat162(ma, mb);
        if (split == SPLIT_BF16_3)
            reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(lo2) + o)[0] = __halves2bfloat162(
                __float2bfloat16_rn(ra - __bfloat162float(ma)), __float2bfloat16_rn(rb - __bfloat162float(mb)));
        return;
    }
    if (split == SPLIT_TF32 || split == SPLIT_TF32_3) {
        const float ha = tf32_rna(va), hb = tf32_rna(vb);
        const float ra = va - ha, rb = vb - hb;  // exact
        const float ma = tf32_rna(ra), mb = tf32_rna(rb);
        reinterpret_cast<float2*>(hi + o)[0] = make_float2(ha, hb);
        reinterpret_cast<float2*>(lo + o)[0] = make_float2(ma, mb);
        if (split == SPLIT_TF32_3) reinterpret_cast<float2*>(lo2 + o)[0] = make_float2(tf32_rna(ra - ma), tf32_rna(rb - mb));
        return;
    }
    if (split == SPLIT_TF32_HI) {
        reinterpret_cast<float2*>(hi + o)[0] = make_float2(tf32_rna(va), tf32_rna(vb));
        return;
    }
    reinterpret_cast<float2*>(hi + o)[0] = make_float2(va, vb);
}

// One warp task is a segment of RX_SEG consecutive points of one grid row
// (RX_SEG / 32 per lane), so that every access is coalesced along the row, all
// loads of a task are issued before its stores, and the only integer divisions
// are two per task, not per point.
constexpr int RX_SEG = 256;
constexpr int RX_PER_LANE = RX_SEG / 32;

// f(t, u) at one point: component values a (u) and b (v), x index, and the y [z]
// factor u0yz of the manufactured solution (ETD_RX_AC_FORCED).
template <typename T, bool FORCED>
__device__ __forceinline__ void rx_eval(const Rx<T>& r, T a, T b, int x, double u0yz, T& f0, T& f1) {
    f0 = (T)0;
    f1 = (T)0;
    switch (r.kind) {
        case ETD_RX_FHN:  // f_u = u - c3 u^3 - v,  f_v = eps (u - a v - b)
            if constexpr (sizeof(T) == 8) {
                // as u (1 - c3 u^2) - v and eps (u - a v) - eps b: five FP64 operations
                // instead of seven (FP64 runs at about two per clock and SM here)
                f0 = fma(a, fma(-r.rp[0], a * a, 1.0), -b);
                f1 = fma(r.rp[1], fma(-r.rp[2], b, a), -(r.rp[1] * r.rp[3]));
            } else {
                f0 = a - r.rp[0] * a * a * a - b;
                f1 = r.rp[1] * (a - r.rp[2] * b - r.rp[3]);
            }
            break;
        case ETD_RX_ALLEN_CAHN:
            f0 = a - a * a * a;
            break;
        case ETD_RX_SINGULAR:
            f0 = r.rp[0] * a / ((T)1 - a);
            break;
        case ETD_RX_AC_FORCED:
            if constexpr (FORCED) {
                // u0 = prod sin(pi x_axis) at x_i = (i+1)/(n+1); psi in FP64
                const double ue = r.decay * u0yz * sinpi((double)(x + 1) / (double)(r.n + 1));
                const double psi = r.psi_coef * ue - ue * (1.0 - ue * ue);
                f0 = (T)((double)a * (1.0 - (double)a * (double)a) + psi);
            }
            break;
        case ETD_RX_LINEAR:
            f0 = r.rp[0] * a;
            f1 = r.rp[0] * b;
            break;
        default:
            if (r.kind < 0) {  // identity: split the field itself
                f0 = a;
                f1 = b;
            }
            break;
    }
}

// FORCED: the manufactured-solution reaction (FP64 forcing term) only; the
// other reactions run in a variant with at most 64 registers per thread (four
// resident blocks of loads in flight per SM instead of three).
template <typename T, bool FORCED>
__global__ void __launch_bounds__(256, FORCED ? 1 : 4) react_kernel(const Rx<T> r) {
    const int lane = threadIdx.x & 31;
    const long long rows_inst = r.npts / r.n;  // n^(d-1) rows per instance
    const int nseg = (r.n + RX_SEG - 1) / RX_SEG;
    const long long tasks = rows_inst * r.ninst * nseg;
    const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
    // pairs of adjacent points per lane (8-byte loads, 4- or 8-byte stores) when
    // every row starts on an even element
    const bool pairs = sizeof(T) == 4 && (r.n % 2 == 0) && (r.ld_in % 2 == 0) && (r.ld_out % 2 == 0) &&
                       (r.bs_in % 2 == 0) && (r.bs_out % 2 == 0);
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tasks; t += wstride) {
        const long long R = t / nseg;
        const int xs = (int)(t - R * nseg) * RX_SEG;  // first point of the segment
        const long long inst = R / rows_inst;
        const long long row = R - inst * rows_inst;
        const T* __restrict__ in = r.in + inst * r.ncomp * r.bs_in + row * r.ld_in;
        const long long oo = inst * r.ncomp * r.bs_out + row * r.ld_out;
        double u0yz = 1.0;  // ETD_RX_AC_FORCED: the y [and z] factors of u0 on this row
        if (FORCED) {
            const double inv = 1.0 / (double)(r.n + 1);
            const long long y = row % r.n, z = row / r.n;
            u0yz = sinpi((double)(y + 1) * inv);
            if (r.d == 3) u0yz *= sinpi((double)(z + 1) * inv);
        }
        if constexpr (sizeof(T) == 4) {
            if (pairs) {
                constexpr int NP = RX_SEG / 64;  // pairs per lane
                float2 u[NP], v[NP];
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const int x = xs + 2 * lane + 64 * j;  // even; x + 1 < n when x < n (n even)
                    const bool ok = x < r.n;
                    u[j] = ok ? reinterpret_cast<const float2*>(in + x)[0] : make_float2(0.f, 0.f);
                    v[j] = (ok && r.ncomp > 1) ? reinterpret_cast<const float2*>(in + r.bs_in + x)[0]
                                               : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const int x = xs + 2 * lane + 64 * j;
                    if (x >= r.n) continue;
                    float fa0, fa1, fb0, fb1;
                    rx_eval<T, FORCED>(r, u[j].x, v[j].x, x, u0yz, fa0, fa1);
                    rx_eval<T, FORCED>(r, u[j].y, v[j].y, x + 1, u0yz, fb0, fb1);
                    // component offsets go into the element index, never into pointer
                    // arithmetic: the operand planes hold 4-byte or 2-byte values
                    store_split2(r.out_hi, r.out_lo, r.out_lo2, oo + x, fa0, fb0, r.split);
                    if (r.ncomp > 1) store_split2(r.out_hi, r.out_lo, r.out_lo2, oo + r.bs_out + x, fa1, fb1, r.split);
                }
                continue;
            }
        }
        T u[RX_PER_LANE], v[RX_PER_LANE];
#pragma unroll
        for (int j = 0; j < RX_PER_LANE; ++j) {
            const int x = xs + lane + 32 * j;
            const bool ok = x < r.n;
            u[j] = ok ? in[x] : (T)0;
            v[j] = (ok && r.ncomp > 1) ? in[r.bs_in + x] : (T)0;
        }
#pragma unroll
        for (int j = 0; j < RX_PER_LANE; ++j) {
            const int x = xs + lane + 32 * j;
            if (x >= r.n) continue;
            T f0, f1;
            rx_eval<T, FORCED>(r, u[j], v[j], x, u0yz, f0, f1);
            store_split(r.out_hi, r.out_lo, r.out_lo2, oo + x, f0, r.split);
            if (r.ncomp > 1) store_split(r.out_hi, r.out_lo, r.out_lo2, oo + r.bs_out + x, f1, r.split);
        }
    }
}

static int grid_for(long long work, int threads) {
    long long blocks = (work + threads - 1) / threads;
    const long long cap = 152LL * 16;  // enough resident blocks to saturate HBM
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// One warp per task, at most the blocks that are resident at once (the warps
// then stride over the tasks; no second wave of blocks).
template <typename T, bool FORCED>
static int react_grid(const Rx<T>& r) {
    static int resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, occ = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, react_kernel<T, FORCED>, 256, 0) != cudaSuccess ||
            sms <= 0 || occ <= 0) {
            sms = 152;
            occ = 4;
        }
        resident = sms * occ;
    }
    const long long tasks = (r.npts / r.n) * r.ninst * ((r.n + RX_SEG - 1) / RX_SEG);
    long long blocks = (tasks + 7) / 8;
    if (blocks > resident) blocks = resident;
    return (int)(blocks < 1 ? 1 : blocks);
}
void launch_react_f32(const Rx<float>& r, cudaStream_t st) {
    if (r.kind == ETD_RX_AC_FORCED)
        react_kernel<float, true><<<react_grid<float, true>(r), 256, 0, st>>>(r);
    else
        react_kernel<float, false><<<react_grid<float, false>(r), 256, 0, st>>>(r);
}
void launch_react_f64(const Rx<double>& r, cudaStream_t st) {
    if (r.kind == ETD_RX_AC_FORCED)
        react_kernel<double, true><<<react_grid<double, true>(r), 256, 0, st>>>(r);
    else
        react_kernel<double, false><<<react_grid<double, false>(r), 256, 0, st>>>(r);
}

// acc[0] = max |u| (as the bit pattern of a non-negative double, so an
// unsigned max is the floating max), acc[1] = number of non-finite entries.
template <typename T>
__global__ void __launch_bounds__(256) stats_kernel(const T* __restrict__ u, long long count,
                                                    unsigned long long* acc) {
    double m = 0.0;
    unsigned long long bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        double v = (double)u[i];
        if (!isfinite(v)) {
            ++bad;
        } else {
            m = fmax(m, fabs(v));
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        bad += __shfl_xor_sync(0xffffffffu, bad, off);
    }
    __shared__ double sm[8];
    __shared__ unsigned long long sb[8];
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    if (l == 0) {
        sm[w] = m;
        sb[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x / 32); ++i) {
            m = fmax(m, sm[i]);
            bad += sb[i];
        }
        atomicMax(&acc[0], (unsigned long long)__double_as_longlong(m));
        if (bad) atomicAdd(&acc[1], bad);
    }
}

// flag |= 1 if the two arrays of `words` 32-bit words differ anywhere (bitwise).
__global__ void __launch_bounds__(256) differ_kernel(const uint4* __restrict__ a, const uint4* __restrict__ b,
                                                     long long n16, const uint32_t* __restrict__ ta,
                                                     const uint32_t* __restrict__ tb, int tail, unsigned* flag) {
    unsigned d = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
        const uint4 x = a[i], y = b[i];
        d |= (x.x ^ y.x) | (x.y ^ y.y) | (x.z ^ y.z) | (x.w ^ y.w);
    }
    if (blockIdx.x == 0 && threadIdx.x < tail) d |= ta[threadIdx.x] ^ tb[threadIdx.x];
    if (__any_sync(0xffffffffu, d != 0) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

void launch_differ(const void* a, const void* b, size_t bytes, unsigned* flag, cudaStream_t st) {
    const long long n16 = (long long)(bytes / 16);
    const int tail = (int)((bytes % 16) / 4);
    const uint32_t* ta = reinterpret_cast<const uint32_t*>(static_cast<const char*>(a) + n16 * 16);
    const uint32_t* tb = reinterpret_cast<const uint32_t*>(static_cast<const char*>(b) + n16 * 16);
    differ_kernel<<<grid_for(n16, 256), 256, 0, st>>>(static_cast<const uint4*>(a), static_cast<const uint4*>(b), n16,
                                                       ta, tb, tail, flag);
}

// One thread: compare the reduced statistics with the bound (step a8).
__global__ void diag_check_kernel(const unsigned long long* __restrict__ acc, double limit, unsigned step,
                                  unsigned* err, double* saved) {
    const double m = __longlong_as_double((long long)acc[0]);
    const unsigned long long bad = acc[1];
    if (bad != 0ull || (limit > 0.0 && m > limit)) {
        if ((atomicOr(err, ERR_DIVERGED) & ERR_DIVERGED) == 0u) {  // the first failure since the last sync
            err[1] = step;
            saved[0] = m;
            saved[1] = (double)bad;
        }
    }
}

void launch_diag_check(const double* acc, double limit, unsigned step, unsigned* err, double* saved,
                       cudaStream_t st) {
    diag_check_kernel<<<1, 1, 0, st>>>(reinterpret_cast<const unsigned long long*>(acc), limit, step, err, saved);
}

void launch_stats_f32(const float* u, long long count, double* acc, cudaStream_t st) {
    stats_kernel<float><<<grid_for(count, 256), 256, 0, st>>>(u, count, (unsigned long long*)acc);
}
void launch_stats_f64(const double* u, long long count, double* acc, cudaStream_t st) {
    stats_kernel<double><<<grid_for(count, 256), 256, 0, st>>>(u, count, (unsigned long long*)acc);
}

}  // namespace etd
