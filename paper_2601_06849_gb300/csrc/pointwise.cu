// Pointwise kernels of the ETD2RK-DS step:
//   - the reaction f(t, u) of all components at one grid point (steps a1 and
//     a5: f(t_n, U) in eq. (13), f(t_{n+1}, W) in eq. (14)), written straight
//     into the operand planes of the next transform pass;
//   - FP64 field diagnostics (step a8): max |u| and the count of non-finite values.
// Both are bandwidth-bound: one read of each component and one write of each
// operand plane per point.
#include "etd_internal.cuh"
#include "../../include/etd.h"

namespace etd {

template <typename T>
__device__ __forceinline__ void store_split(T* hi, T* lo, T* lo2, long long o, T v, int split) {
    if constexpr (sizeof(T) == 4) {
        if (split == SPLIT_BF16_2 || split == SPLIT_BF16_3) {
            split_bf16((double)v, split == SPLIT_BF16_3 ? 3 : 2, reinterpret_cast<__nv_bfloat16*>(hi),
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

template <typename T>
__global__ void __launch_bounds__(256) react_kernel(const Rx<T> r) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long total = r.npts * r.ninst;
    for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < total; pt += stride) {
        const long long inst = pt / r.npts;
        const long long p = pt - inst * r.npts;
        const long long row = p / r.n;
        const int x = (int)(p - row * r.n);
        const long long oi = inst * r.ncomp * r.bs_in + row * r.ld_in + x;
        const long long oo = inst * r.ncomp * r.bs_out + row * r.ld_out + x;
        switch (r.kind) {
            case ETD_RX_FHN: {
                // f_u = u - c3 u^3 - v,  f_v = eps (u - a v - b)
                const T u = r.in[oi], v = r.in[r.bs_in + oi];
                // component offsets go into the element index, never into pointer
                // arithmetic: the operand planes hold 4-byte or 2-byte values
                store_split(r.out_hi, r.out_lo, r.out_lo2, oo, u - r.rp[0] * u * u * u - v, r.split);
                store_split(r.out_hi, r.out_lo, r.out_lo2, oo + r.bs_out, r.rp[1] * (u - r.rp[2] * v - r.rp[3]),
                            r.split);
                break;
            }
            case ETD_RX_ALLEN_CAHN: {
                const T u = r.in[oi];
                store_split(r.out_hi, r.out_lo, r.out_lo2, oo, u - u * u * u, r.split);
                break;
            }
            case ETD_RX_SINGULAR: {
                const T u = r.in[oi];
                store_split(r.out_hi, r.out_lo, r.out_lo2, oo, r.rp[0] * u / ((T)1 - u), r.split);
                break;
            }
            case ETD_RX_AC_FORCED: {
                // u0 = prod sin(pi x_axis) at x_i = (i+1)/(n+1); psi in FP64
                const double inv = 1.0 / (double)(r.n + 1);
                const long long y = row % r.n, z = row / r.n;
                double u0 = sinpi((double)(x + 1) * inv) * sinpi((double)(y + 1) * inv);
                if (r.d == 3) u0 *= sinpi((double)(z + 1) * inv);
                const double ue = r.decay * u0;
                const double psi = r.psi_coef * ue - ue * (1.0 - ue * ue);
                const T u = r.in[oi];
                store_split(r.out_hi, r.out_lo, r.out_lo2, oo, (T)((double)u * (1.0 - (double)u * (double)u) + psi),
                            r.split);
                break;
            }
            default:
                for (int c = 0; c < r.ncomp; ++c) {
                    const T u = r.in[c * r.bs_in + oi];
                    T f = (T)0;
                    if (r.kind == ETD_RX_LINEAR) f = r.rp[0] * u;
                    else if (r.kind < 0) f = u;  // identity: split the field itself
                    store_split(r.out_hi, r.out_lo, r.out_lo2, oo + c * r.bs_out, f, r.split);
                }
                break;
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

void launch_react_f32(const Rx<float>& r, cudaStream_t st) {
    react_kernel<float><<<grid_for(r.npts * r.ninst, 256), 256, 0, st>>>(r);
}
void launch_react_f64(const Rx<double>& r, cudaStream_t st) {
    react_kernel<double><<<grid_for(r.npts * r.ninst, 256), 256, 0, st>>>(r);
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

void launch_stats_f32(const float* u, long long count, double* acc, cudaStream_t st) {
    stats_kernel<float><<<grid_for(count, 256), 256, 0, st>>>(u, count, (unsigned long long*)acc);
}
void launch_stats_f64(const double* u, long long count, double* acc, cudaStream_t st) {
    stats_kernel<double><<<grid_for(count, 256), 256, 0, st>>>(u, count, (unsigned long long*)acc);
}

}  // namespace etd
