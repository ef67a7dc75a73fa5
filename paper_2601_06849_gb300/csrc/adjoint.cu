// Kernels of the adjoint step (reverse-mode derivative of eq. (13)-(16)).
// With S = E1(tau A_2) [E1(tau A_2^z)] and X_l = E_l(tau A_1), symmetric and
// commuting, and everything diagonal in the eigenbasis:
//   Gbar = tau X3 U+bar;  Wbar = U+bar + J_f(W)^T Gbar;
//   Fbar = tau X2 S Wbar - S Gbar;  Ubar = X1 S Wbar + J_f(U)^T Fbar,
//   dL/dkappa_c = sum over modes of [ U+bar^ d(tau E3) G^ - Gbar^ dS F^
//                 + Wbar^ (d(E1 S) U^ + d(tau E2 S) F^) ],  G^ = F_W^ - S F^,
//   dL/dtheta = <Gbar, d_theta f(W)> + <Fbar, d_theta f(U)>.
// Fields here use the caller's layout (rows of n, no padding); spectral arrays
// are [comp][p][l][k] with k the x mode.
#include <type_traits>

#include "../../include/etd.h"
#include "etd_internal.cuh"

namespace etd {

namespace {

__device__ __forceinline__ double xfactor(const double* g, int n, int sel, int k) {
    return sel == 0 ? 1.0 : g[(sel - 1) * n + k];  // 1: E1, 2: tau E2, 3: tau E3
}

// The spectral kernels walk one row (l, p) of n x modes per warp, lanes along k:
// the row's y [z] factors and its index arithmetic are formed once per row, and
// every access is coalesced. GB300 runs FP64 at a small fraction of its FP32
// rate, so the FP32 paths (T = float: inputs and outputs in FP32, each with the
// relative error of the transforms that made it) form the per-point products in
// FP32 from the double-float factor grids and accumulate the gradient sums in
// FP64 per row; the FP64 path computes in FP64 throughout.
#define ETD_FOR_ROWS(npts, n)                                                                                      \
    const long long rows_ = (npts) / (n);                                                                          \
    const long long wstride_ = (long long)gridDim.x * (blockDim.x >> 5);                                            \
    for (long long row = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows_; row += wstride_)

template <typename T>
__global__ void __launch_bounds__(256) spec_combine_kernel(SpecCombine<T> a) {
    const int c = blockIdx.y, lane = threadIdx.x & 31;
    ETD_FOR_ROWS(a.npts, a.n) {
        const int l = (int)(row % a.n), p = (int)(row / a.n);  // p = 0 in 2D
        const long long base = (long long)c * a.npts + row * a.n;
        if constexpr (sizeof(T) == 4) {
            // The mode factors X_k S are applied again at every step of the window, so
            // they are formed as double-floats: an FP32 factor would repeat its
            // rounding error at every step (about n_steps 2^-24 after n_steps); the
            // only FP32 rounding left is that of each output value.
            const float2* g = a.grid2 + (long long)c * 3 * a.n;
            const float2 one = make_float2(1.f, 0.f);
            const float2 s = (a.d == 2) ? g[l] : ff_mul(g[l], g[p]);
            const float2 s1 = a.s1 ? s : one, s2 = a.s2 ? s : one;
            const float sa = (float)a.alpha, sb = (float)a.beta;  // 1, -1 or 0: exact in FP32
            for (int k = lane; k < a.n; k += 32) {
                float2 v = make_float2(0.f, 0.f);
                if (a.in1) {
                    const float2 x = a.xsel1 ? g[(a.xsel1 - 1) * a.n + k] : one;
                    v = ff_mul_f(ff_mul(x, s1), sa * a.in1[base + k]);
                }
                if (a.in2) {
                    const float2 x = a.xsel2 ? g[(a.xsel2 - 1) * a.n + k] : one;
                    v = ff_add(v, ff_mul_f(ff_mul(x, s2), sb * a.in2[base + k]));
                }
                a.out[base + k] = __fadd_rn(v.x, v.y);
            }
        } else {
            const double* g = a.grid + (long long)c * 3 * a.n;
            const double s = (a.d == 2) ? g[l] : g[l] * g[p];
            for (int k = lane; k < a.n; k += 32) {
                double v = 0.0;
                if (a.in1) v += a.alpha * xfactor(g, a.n, a.xsel1, k) * (a.s1 ? s : 1.0) * (double)a.in1[base + k];
                if (a.in2) v += a.beta * xfactor(g, a.n, a.xsel2, k) * (a.s2 ? s : 1.0) * (double)a.in2[base + k];
                a.out[base + k] = (T)v;
            }
        }
    }
}

// out = base + J_f(X)^T V at every point (all components of a point at once)
template <typename T>
__global__ void react_vjp_kernel(ReactVjp<T> a) {
    using C = typename std::conditional<sizeof(T) == 4, float, double>::type;  // compute type
    const C c3 = (C)a.rp[0], rp1 = (C)a.rp[1], rp2 = (C)a.rp[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.npts;
         i += (long long)gridDim.x * blockDim.x) {
        switch (a.kind) {
            case ETD_RX_FHN: {  // rp = (c3, eps, a, b)
                const C u = a.X[i], v0 = a.V[i], v1 = a.V[a.npts + i];
                a.out[i] = (T)((C)a.base[i] + ((C)1 - (C)3 * c3 * u * u) * v0 + rp1 * v1);
                a.out[a.npts + i] = (T)((C)a.base[a.npts + i] - v0 - rp1 * rp2 * v1);
                break;
            }
            default:
                for (int c = 0; c < a.ncomp; ++c) {
                    const long long o = c * a.npts + i;
                    const C x = a.X[o];
                    C j = 0;
                    if (a.kind == ETD_RX_LINEAR) j = c3;
                    else if (a.kind == ETD_RX_ALLEN_CAHN) j = (C)1 - (C)3 * x * x;
                    else if (a.kind == ETD_RX_SINGULAR) j = c3 / (((C)1 - x) * ((C)1 - x));
                    a.out[o] = (T)((C)a.base[o] + j * (C)a.V[o]);
                }
                break;
        }
    }
}

__device__ __forceinline__ void block_add(double v, double* target) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __shared__ double sm[32];
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += sm[i];
        atomicAdd(target, t);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) grad_kappa_kernel(GradKappa<T> a) {
    const int c = blockIdx.y, lane = threadIdx.x & 31;
    double acc = 0.0;
    ETD_FOR_ROWS(a.npts, a.n) {
        const int l = (int)(row % a.n), p = (int)(row / a.n);
        const long long base = (long long)c * a.npts + row * a.n;
        if constexpr (sizeof(T) == 4) {
            const float2* g = a.grid2 + (long long)c * 3 * a.n;
            const float2* dg = a.dgrid2 + (long long)c * 3 * a.n;
            // s = S as a double-float (G^ = F_W^ - S F^ cancels), ds = dS/dkappa in FP32
            const float2 s = (a.d == 2) ? g[l] : ff_mul(g[l], g[p]);
            const float ds = (a.d == 2) ? dg[l].x : fmaf(dg[l].x, g[p].x, __fmul_rn(g[l].x, dg[p].x));
            for (int k0 = lane; k0 < a.n; k0 += 4 * 32) {
                float part = 0.f;  // at most four of this lane's terms in FP32, then FP64
                for (int k = k0; k < a.n && k < k0 + 4 * 32; k += 32) {
                    const long long o = base + k;
                    const float fh = a.Fh[o], uh = a.Uh[o], wb = a.Wbh[o];
                    const float gh = fmaf(-s.y, fh, fmaf(-s.x, fh, a.FWh[o]));
                    const float e1 = fmaf(dg[k].x, s.x, __fmul_rn(g[k].x, ds));                  // d(E1 S)
                    const float e2 = fmaf(dg[a.n + k].x, s.x, __fmul_rn(g[a.n + k].x, ds));      // d(tau E2 S)
                    part += __fmul_rn(a.Lh[o], dg[2 * a.n + k].x) * gh - __fmul_rn(a.Gbh[o], ds) * fh +
                            wb * fmaf(e1, uh, __fmul_rn(e2, fh));
                }
                acc += (double)part;
            }
        } else {
            const double* g = a.grid + (long long)c * 3 * a.n;
            const double* dg = a.dgrid + (long long)c * 3 * a.n;
            double s, ds;
            if (a.d == 2) {
                s = g[l];
                ds = dg[l];
            } else {
                s = g[l] * g[p];
                ds = dg[l] * g[p] + g[l] * dg[p];
            }
            for (int k = lane; k < a.n; k += 32) {
                const long long o = base + k;
                const double fh = a.Fh[o], uh = a.Uh[o];
                const double gh = (double)a.FWh[o] - s * fh;
                const double wb = a.Wbh[o];
                acc += (double)a.Lh[o] * dg[2 * a.n + k] * gh - (double)a.Gbh[o] * ds * fh +
                       wb * ((dg[k] * s + g[k] * ds) * uh + (dg[a.n + k] * s + g[a.n + k] * ds) * fh);
            }
        }
    }
    block_add(acc, a.out + c);
}

template <typename T>
__global__ void __launch_bounds__(256) grad_rx_kernel(GradRx<T> a) {
    using C = typename std::conditional<sizeof(T) == 4, float, double>::type;  // per-point compute type
    // per point in the compute type, at most four points per partial sum, the
    // partial sums in FP64
    C g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    double d0 = 0, d1 = 0, d2 = 0, d3 = 0;
    int cnt = 0;
    const C eps = (C)a.rp[1], aa = (C)a.rp[2], bb = (C)a.rp[3];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.npts;
         i += (long long)gridDim.x * blockDim.x) {
        if (cnt == 4) {
            d0 += (double)g0;
            d1 += (double)g1;
            d2 += (double)g2;
            d3 += (double)g3;
            g0 = g1 = g2 = g3 = 0;
            cnt = 0;
        }
        ++cnt;
        if (a.kind == ETD_RX_FHN) {
            const C wu = a.W[i], wv = a.W[a.npts + i], uu = a.U[i], uv = a.U[a.npts + i];
            const C gbu = a.Gb[i], gbv = a.Gb[a.npts + i], fbu = a.Fb[i], fbv = a.Fb[a.npts + i];
            g0 += -gbu * wu * wu * wu - fbu * uu * uu * uu;
            g1 += gbv * (wu - aa * wv - bb) + fbv * (uu - aa * uv - bb);
            g2 += -eps * (gbv * wv + fbv * uv);
            g3 += -eps * (gbv + fbv);
        } else if (a.kind == ETD_RX_LINEAR) {
            for (int c = 0; c < a.ncomp; ++c) {
                const long long o = c * a.npts + i;
                g0 += (C)a.Gb[o] * (C)a.W[o] + (C)a.Fb[o] * (C)a.U[o];
            }
        } else if (a.kind == ETD_RX_SINGULAR) {
            const C w = a.W[i], u = a.U[i];
            g0 += (C)a.Gb[i] * w / ((C)1 - w) + (C)a.Fb[i] * u / ((C)1 - u);
        }
    }
    block_add(d0 + (double)g0, a.out + 0);
    block_add(d1 + (double)g1, a.out + 1);
    block_add(d2 + (double)g2, a.out + 2);
    block_add(d3 + (double)g3, a.out + 3);
}

int blocks_for(long long work) {
    long long b = (work + 255) / 256;
    if (b > 152LL * 8) b = 152LL * 8;
    return (int)(b < 1 ? 1 : b);
}

// Blocks for the kernels that give one warp to each spectral row of n modes
// (eight rows per 256-thread block): a grid sized by points would leave most
// warps without a row.
int blocks_for_rows(long long npts, int n) {
    return blocks_for((npts / n) * 32);
}

}  // namespace

template <typename T>
void launch_spec_combine(const SpecCombine<T>& a, cudaStream_t st) {
    spec_combine_kernel<T><<<dim3(blocks_for_rows(a.npts, a.n), a.ncomp), 256, 0, st>>>(a);
}
template <typename T>
void launch_react_vjp(const ReactVjp<T>& a, cudaStream_t st) {
    react_vjp_kernel<T><<<blocks_for(a.npts), 256, 0, st>>>(a);
}
template <typename T>
void launch_grad_kappa(const GradKappa<T>& a, cudaStream_t st) {
    grad_kappa_kernel<T><<<dim3(blocks_for_rows(a.npts, a.n), a.ncomp), 256, 0, st>>>(a);
}
template <typename T>
void launch_grad_rx(const GradRx<T>& a, cudaStream_t st) {
    grad_rx_kernel<T><<<blocks_for(a.npts), 256, 0, st>>>(a);
}

template void launch_spec_combine<float>(const SpecCombine<float>&, cudaStream_t);
template void launch_spec_combine<double>(const SpecCombine<double>&, cudaStream_t);
template void launch_react_vjp<float>(const ReactVjp<float>&, cudaStream_t);
template void launch_react_vjp<double>(const ReactVjp<double>&, cudaStream_t);
template void launch_grad_kappa<float>(const GradKappa<float>&, cudaStream_t);
template void launch_grad_kappa<double>(const GradKappa<double>&, cudaStream_t);
template void launch_grad_rx<float>(const GradRx<float>&, cudaStream_t);
template void launch_grad_rx<double>(const GradRx<double>&, cudaStream_t);

}  // namespace etd
