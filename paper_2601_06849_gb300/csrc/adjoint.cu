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
#include "../../include/etd.h"
#include "etd_internal.cuh"

namespace etd {

namespace {

__device__ __forceinline__ double xfactor(const double* g, int n, int sel, int k) {
    return sel == 0 ? 1.0 : g[(sel - 1) * n + k];  // 1: E1, 2: tau E2, 3: tau E3
}

__device__ __forceinline__ void spectral_index(long long idx, int n, int d, int& k, int& l, int& p) {
    k = (int)(idx % n);
    const long long r = idx / n;
    l = (int)(r % n);
    p = (d == 3) ? (int)(r / n) : -1;
}

template <typename T>
__global__ void spec_combine_kernel(SpecCombine<T> a) {
    const long long total = a.npts * a.ncomp;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i / a.npts);
        int k, l, p;
        spectral_index(i - c * a.npts, a.n, a.d, k, l, p);
        const double* g = a.grid + (long long)c * 3 * a.n;
        const double s = (a.d == 2) ? g[l] : g[l] * g[p];
        double v = 0.0;
        if (a.in1) v += a.alpha * xfactor(g, a.n, a.xsel1, k) * (a.s1 ? s : 1.0) * (double)a.in1[i];
        if (a.in2) v += a.beta * xfactor(g, a.n, a.xsel2, k) * (a.s2 ? s : 1.0) * (double)a.in2[i];
        a.out[i] = (T)v;
    }
}

// out = base + J_f(X)^T V at every point (all components of a point at once)
template <typename T>
__global__ void react_vjp_kernel(ReactVjp<T> a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.npts;
         i += (long long)gridDim.x * blockDim.x) {
        switch (a.kind) {
            case ETD_RX_FHN: {
                const double u = a.X[i], v0 = a.V[i], v1 = a.V[a.npts + i];
                const double c3 = a.rp[0], eps = a.rp[1], aa = a.rp[2];
                a.out[i] = (T)((double)a.base[i] + (1.0 - 3.0 * c3 * u * u) * v0 + eps * v1);
                a.out[a.npts + i] = (T)((double)a.base[a.npts + i] - v0 - eps * aa * v1);
                break;
            }
            default:
                for (int c = 0; c < a.ncomp; ++c) {
                    const long long o = c * a.npts + i;
                    const double x = a.X[o];
                    double j = 0.0;
                    if (a.kind == ETD_RX_LINEAR) j = a.rp[0];
                    else if (a.kind == ETD_RX_ALLEN_CAHN) j = 1.0 - 3.0 * x * x;
                    else if (a.kind == ETD_RX_SINGULAR) j = a.rp[0] / ((1.0 - x) * (1.0 - x));
                    a.out[o] = (T)((double)a.base[o] + j * (double)a.V[o]);
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
    const int c = blockIdx.y;
    const double* g = a.grid + (long long)c * 3 * a.n;
    const double* dg = a.dgrid + (long long)c * 3 * a.n;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.npts;
         i += (long long)gridDim.x * blockDim.x) {
        int k, l, p;
        spectral_index(i, a.n, a.d, k, l, p);
        const long long o = c * a.npts + i;
        double s, ds;
        if (a.d == 2) {
            s = g[l];
            ds = dg[l];
        } else {
            s = g[l] * g[p];
            ds = dg[l] * g[p] + g[l] * dg[p];
        }
        const double fh = a.Fh[o], uh = a.Uh[o];
        const double gh = (double)a.FWh[o] - s * fh;
        const double wb = a.Wbh[o];
        acc += (double)a.Lh[o] * dg[2 * a.n + k] * gh - (double)a.Gbh[o] * ds * fh +
               wb * ((dg[k] * s + g[k] * ds) * uh + (dg[a.n + k] * s + g[a.n + k] * ds) * fh);
    }
    block_add(acc, a.out + c);
}

template <typename T>
__global__ void __launch_bounds__(256) grad_rx_kernel(GradRx<T> a) {
    double g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.npts;
         i += (long long)gridDim.x * blockDim.x) {
        if (a.kind == ETD_RX_FHN) {
            const double eps = a.rp[1], aa = a.rp[2], bb = a.rp[3];
            const double wu = a.W[i], wv = a.W[a.npts + i], uu = a.U[i], uv = a.U[a.npts + i];
            const double gbu = a.Gb[i], gbv = a.Gb[a.npts + i], fbu = a.Fb[i], fbv = a.Fb[a.npts + i];
            g0 += -gbu * wu * wu * wu - fbu * uu * uu * uu;
            g1 += gbv * (wu - aa * wv - bb) + fbv * (uu - aa * uv - bb);
            g2 += -eps * (gbv * wv + fbv * uv);
            g3 += -eps * (gbv + fbv);
        } else if (a.kind == ETD_RX_LINEAR) {
            for (int c = 0; c < a.ncomp; ++c) {
                const long long o = c * a.npts + i;
                g0 += (double)a.Gb[o] * a.W[o] + (double)a.Fb[o] * a.U[o];
            }
        } else if (a.kind == ETD_RX_SINGULAR) {
            const double w = a.W[i], u = a.U[i];
            g0 += (double)a.Gb[i] * w / (1.0 - w) + (double)a.Fb[i] * u / (1.0 - u);
        }
    }
    block_add(g0, a.out + 0);
    block_add(g1, a.out + 1);
    block_add(g2, a.out + 2);
    block_add(g3, a.out + 3);
}

int blocks_for(long long work) {
    long long b = (work + 255) / 256;
    if (b > 152LL * 8) b = 152LL * 8;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
void launch_spec_combine(const SpecCombine<T>& a, cudaStream_t st) {
    spec_combine_kernel<T><<<blocks_for(a.npts * a.ncomp), 256, 0, st>>>(a);
}
template <typename T>
void launch_react_vjp(const ReactVjp<T>& a, cudaStream_t st) {
    react_vjp_kernel<T><<<blocks_for(a.npts), 256, 0, st>>>(a);
}
template <typename T>
void launch_grad_kappa(const GradKappa<T>& a, cudaStream_t st) {
    grad_kappa_kernel<T><<<dim3(blocks_for(a.npts), a.ncomp), 256, 0, st>>>(a);
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
