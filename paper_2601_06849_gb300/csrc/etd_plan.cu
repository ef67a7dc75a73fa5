// Host side of the ETD2RK-DS library: plan precompute, step orchestration and
// the C ABI declared in include/etd.h.
//
// Plan (Algorithm 1/2, steps 1-2, done once in FP64 on the host):
//   - A_x = (1/h^2) tridiag(-kappa, 2 kappa + (q/d) h^2, -kappa) has the
//     orthonormal sine eigenvectors P[j][k] = sqrt(2/(n+1)) sin(pi (j+1)(k+1)/(n+1))
//     and eigenvalues lambda_k = (4 kappa/h^2) sin^2(pi (k+1)/(2(n+1))) + q/d
//     (Section 3.3.2 uses A_x = P_x D_x P_x^T; with equal spacing on every axis
//     P_x = P_y = P_z and only lambda depends on the component's kappa);
//   - the factor grids E_l(tau lambda_k), l = 1, 2, 3, of the chosen family:
//     Q_l of Section 3.1 (P_{0,2}), R_l of Section 5 (P_{0,4}), or the exact
//     exponential functions of eq. (9)-(10). Algorithm 1 stores
//     d^(l) = Re(r_l / (tau lambda - s)); the real rational E_l = 2 d^(l) is
//     evaluated directly instead.
//
// Step (eq. (13)-(16) in the eigenbasis, where every operator is diagonal; the
// spectral coefficients U^ of u are carried from step to step):
//   F = f(t_n, U)                                      reaction kernel
//   F^ = T(F);  W^ = E1x E1y.. U^ + tau E2x E1y.. F^   d passes, last one fused
//   W = T(W^)                                          d passes
//   F_W = f(t_{n+1}, W)                                reaction kernel
//   F_W^ = T(F_W); U^+ = W^ + tau E3x (F_W^ - E1y.. F^) d passes, last one fused
//   U+ = T(U^+)                                        d passes
// T is its own inverse (P symmetric orthogonal), so every pass is the same
// product with P. 4d passes of 2 n^(d+1) flops: 16 n flops per unknown in 2D,
// 24 n in 3D.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <string>
#include <vector>

#include "../../include/etd.h"
#include "etd_internal.cuh"

using namespace etd;

struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
};

struct etd_plan {
    int d = 0, n = 0, ncomp = 1, precision = ETD_PREC_BF16X6, pade = 2, reaction = ETD_RX_ALLEN_CAHN;
    int ninst = 1;  // instances stepped together (same d and n); batch index = instance * ncomp + comp
    double rp[8] = {0};
    double kappa[2] = {0, 0};
    double q = 0, tau = 0, t = 0;
    cudaStream_t stream = nullptr;
    int M = 0, mq = 0, ld = 0;
    long long bs = 0, npts = 0;
    size_t elem = 4;
    bool use_tc = false;
    bool dst = false;         // ETD_PREC_DST32: FFT-based sine transforms instead of products with P
    float2* dst_tw = nullptr; // its FFT twiddles by stage (N - 1 of them, N = 2(n+1))
    void* dst_tmp = nullptr;  // its natural-order scratch rows
    bool ozaki = false;       // ETD_PREC_FP64_SPLIT*: FP64 products as exact BF16 slice products
    int oz_s = 0;             // its slice count (6, 5 or 4)
    void* oz_slices[OZ_S] = {nullptr};  // the operand's BF16 slices (one set, refilled before every pass)
    void* oz_P[OZ_S] = {nullptr};       // P's slices
    int* oz_rexp = nullptr;             // per operand row: the slices' scale exponent
    int oz_pexp = 0;                    // P's scale exponent
    bool bf16 = false;  // BF16 operand pieces (ETD_PREC_BF16X3 / X6)
    size_t op_elem = 4; // bytes per operand-plane value
    int pieces = 1;     // operand planes allocated per buffer
    int out_slot = 0;   // config slot of the transform that returns the field
    // device memory
    void* P[3] = {nullptr, nullptr, nullptr};  // pieces of the sine basis
    void* grid = nullptr;   // FP64 factor grids [comp][3][n]
    void* grid2 = nullptr;  // the same as double-floats (FP32 paths)
    void* uhat = nullptr;
    void* zhat = nullptr;  // Z between the two stages of a step
    void* wphys = nullptr;
    void* op[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // operand buffers x pieces
    unsigned* err = nullptr;
    double* stats = nullptr;  // [0..1] reductions, [3] etd_step_host's compare flag, [4..5] first failed check
    int diag_every = 0;       // in-step field check every diag_every steps (0 = off)
    double diag_max = 0;      // bound on max |u| of that check (<= 0: non-finite values only)
    long long steps_done = 0; // time steps taken over the plan's life (the check's counter)
    void* host_field = nullptr;  // etd_step_host: the field being stepped (the last one returned)
    void* host_in = nullptr;     // etd_step_host: the incoming field
    bool host_valid = false;     // host_field holds the field the last etd_step_host returned
    void* host_snap = nullptr;   // etd_step_host: a device copy of the field the last call returned
    cudaStream_t copy_stream = nullptr;  // etd_step_host: the input's copy and comparison beside the step
    cudaEvent_t ev_host = nullptr;
    cudaStream_t out_stream[3] = {};     // etd_step_host: three of the four parts of the result's copy out
    cudaEvent_t ev_out[4] = {};
    long long workspace = 0;
    // carried spectral state
    bool uhat_valid = false;
    const void* uhat_src = nullptr;
    // fused reaction (rx_fusable): the last step's final epilogue left the operand
    // pieces of f(U) for the next step in op[rx_cur] (for the field rx_src)
    bool rx_ready = false;
    int rx_cur = 0;
    const void* rx_src = nullptr;
    // tensor-core pass: slot 0 = every internal pass, slot 1 = the output transform
    TcConfig tc[2] = {};
    TcMaps* maps = nullptr;
    // timing
    bool timing = false;
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> pool;
    // ensemble container (etd_batch_create): one group plan per distinct (d, n)
    bool is_batch = false;
    std::vector<etd_plan*> groups;
    std::vector<std::vector<int>> members;  // instance indices of each group
    std::vector<void*> gfield;              // contiguous fields of each group
    std::vector<const void*> last_ptrs;     // u_dev of the previous etd_batch_step
    cudaEvent_t ev_start = nullptr;
    std::vector<cudaEvent_t> ev_done;
    long long count = 0;
    cudaGraphExec_t step_graph = nullptr;  // one inner step of every group (not the last of a call)
    // adjoint workspace (etd_step_adjoint), allocated on first use
    std::vector<void*> adj_traj;  // forward states of the window being differentiated
    void* adj_work[14] = {nullptr};
    double* adj_dgrid = nullptr;  // kappa derivatives of E1, tau E2, tau E3 per component
    float2* adj_dgrid2 = nullptr;  // the same as double-floats (FP32 paths)
    double* adj_acc = nullptr;    // [2] kappa gradients, [4] reaction-parameter gradients
    cudaStream_t cap_stream = nullptr;      // capture origin (the caller's stream may be the legacy one)
};

namespace {

thread_local std::string g_last_error;

etd_status fail(etd_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

#define ETD_CUDA(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(ETD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// E_1, E_2, E_3 at x = tau * lambda >= 0 in FP64.
void factor_grids(int family, double x, double* e) {
    if (family == ETD_PADE_02) {
        const double den = x * x + 2 * x + 2;
        e[0] = 2 / den;
        e[1] = (x + 2) / den;
        e[2] = (x + 1) / den;
    } else if (family == ETD_PADE_04) {
        const double den = (((x + 4) * x + 12) * x + 24) * x + 24;
        e[0] = 24 / den;
        e[1] = (((x + 4) * x + 12) * x + 24) / den;
        e[2] = (((x + 3) * x + 8) * x + 12) / den;
    } else {
        // e^{-x}, (1 - e^{-x})/x, (x - 1 + e^{-x})/x^2; series where x - 1 + e^{-x} cancels
        e[0] = std::exp(-x);
        e[1] = (x > 0) ? -std::expm1(-x) / x : 1.0;
        if (x < 0.05) {
            double term = 0.5, sum = 0.0;  // sum_{j>=0} (-x)^j / (j+2)!
            for (int j = 0; j < 10; ++j) {
                sum += term;
                term *= -x / (double)(j + 3);
            }
            e[2] = sum;
        } else {
            e[2] = (x + std::expm1(-x)) / (x * x);
        }
    }
}

// Round to BF16 (7 stored mantissa bits), nearest with ties to even: add half an
// ulp of the kept part (minus one when the kept part is even) and truncate.
uint16_t bf16_round_host(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_to_float_host(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Round to TF32 (10 stored mantissa bits), nearest with ties away from zero.
float tf32_round_host(float v) {
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return v;
    u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

etd_status dalloc(etd_plan* p, void** ptr, size_t bytes) {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? ETD_ERR_OOM : ETD_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    p->workspace += (long long)bytes;
    return ETD_OK;
}

void free_plan(etd_plan* p) {
    for (etd_plan* g : p->groups) {
        if (g->stream) cudaStreamDestroy(g->stream);
        free_plan(g);
    }
    for (void* f : p->gfield)
        if (f) cudaFree(f);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->step_graph) cudaGraphExecDestroy(p->step_graph);
    for (void* f : p->adj_traj)
        if (f) cudaFree(f);
    for (void* f : p->adj_work)
        if (f) cudaFree(f);
    if (p->adj_dgrid) cudaFree(p->adj_dgrid);
    if (p->adj_dgrid2) cudaFree(p->adj_dgrid2);
    if (p->adj_acc) cudaFree(p->adj_acc);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->ev_host) cudaEventDestroy(p->ev_host);
    for (cudaStream_t& st : p->out_stream)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t& ev : p->ev_out)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : p->ev_done)
        if (ev) cudaEventDestroy(ev);
    void* bufs[] = {p->P[0],     p->P[1],     p->P[2],     p->grid,     p->grid2,    p->uhat,     p->zhat,
                    p->wphys,    p->op[0][0], p->op[0][1], p->op[0][2], p->op[1][0],
                    p->op[1][1], p->op[1][2], p->err,      p->stats,    p->host_field, p->host_in,
                    p->dst_tw,   p->dst_tmp,  p->host_snap};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (p->maps) tc_maps_destroy(p->maps);
    for (int i = 0; i < OZ_S; ++i) {
        if (p->oz_slices[i]) cudaFree(p->oz_slices[i]);
        if (p->oz_P[i]) cudaFree(p->oz_P[i]);
    }
    if (p->oz_rexp) cudaFree(p->oz_rexp);
    for (auto& tl : p->timed) {
        cudaEventDestroy(tl.a);
        cudaEventDestroy(tl.b);
    }
    for (auto ev : p->pool) cudaEventDestroy(ev);
    delete p;
}

cudaEvent_t take_event(etd_plan* p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct TimerScope {
    etd_plan* p;
    int kind;
    cudaEvent_t a = nullptr;
    TimerScope(etd_plan* pp, int k) : p(pp), kind(k) {
        if (p->timing) {
            a = take_event(p);
            cudaEventRecord(a, p->stream);
        }
    }
    ~TimerScope() {
        if (p->timing) {
            cudaEvent_t b = take_event(p);
            cudaEventRecord(b, p->stream);
            p->timed.push_back({kind, a, b});
        }
    }
};

template <typename T>
Epi<T> base_epi(const etd_plan* p) {
    Epi<T> e{};
    e.d = p->d;
    e.n = p->n;
    e.M = p->M;
    e.mq = p->mq;
    e.ld = p->ld;
    e.bs = p->bs;
    using St = typename Epi<T>::St;
    e.uhat = (St*)p->uhat;
    e.zhat = (St*)p->zhat;
    e.grid = (const St*)(sizeof(T) == 4 ? p->grid2 : p->grid);
    return e;
}

int split_for(const etd_plan* p, int slot) {
    if (!p->use_tc) return SPLIT_NONE;
    const int pieces = p->tc[slot].pieces;
    if (p->bf16) return pieces == 3 ? SPLIT_BF16_3 : SPLIT_BF16_2;
    return pieces == 3 ? SPLIT_TF32_3 : (pieces == 2 ? SPLIT_TF32 : SPLIT_TF32_HI);
}

// One pass reading operand buffer `cur` with the products of config `slot`; the
// epilogue's operand output (if any) goes to buffer 1 - cur split as `out_split`.
template <typename T>
etd_status run_pass(etd_plan* p, int cur, int slot, int mode, int out_split, void* dst, int ld_dst,
                    long long bs_dst) {
    Epi<T> e = base_epi<T>(p);
    e.mode = mode;
    e.split = out_split;
    e.op_hi = (T*)p->op[1 - cur][0];
    e.op_lo = (T*)p->op[1 - cur][1];
    e.op_lo2 = (T*)p->op[1 - cur][2];
    e.dst = (T*)dst;
    e.ld_dst = ld_dst;
    e.bs_dst = bs_dst;
    e.rx = p->reaction;
    e.rx_c = (T)p->rp[0];
    TimerScope ts(p, slot == p->out_slot && p->out_slot != 0 ? 2 : 0);
    if constexpr (sizeof(T) == 8) {
        if (p->ozaki) {
            cudaError_t ce = launch_ozaki_pass(p->oz_s, p->oz_P, p->oz_pexp, (const double*)p->op[cur][0], p->M, p->n,
                                               p->ninst * p->ncomp, p->ld, p->oz_slices, p->oz_rexp, e, p->err,
                                               p->stream);
            if (ce != cudaSuccess) return fail(ETD_ERR_CUDA, "FP64-split pass launch: %s", cudaGetErrorString(ce));
            return ETD_OK;
        }
        launch_gemm_simt_f64((const double*)p->op[cur][0], (const double*)p->P[0], p->M, p->n, p->ninst * p->ncomp,
                             e, p->stream);
    } else {
        if (p->use_tc) {
            cudaError_t ce =
                launch_gemm_tc(p->tc[slot], slot, p->maps, cur, p->M, p->n, p->ninst * p->ncomp, e, p->err, p->stream);
            if (ce != cudaSuccess) return fail(ETD_ERR_CUDA, "tensor-core pass launch: %s", cudaGetErrorString(ce));
            return ETD_OK;
        }
        if (p->dst) {
            cudaError_t ce = launch_dst_pass((const float*)p->op[cur][0], p->M, p->n, p->ninst * p->ncomp, p->ld,
                                             p->bs, p->dst_tw, (float*)p->dst_tmp, e, p->stream);
            if (ce != cudaSuccess) return fail(ETD_ERR_CUDA, "sine transform pass: %s", cudaGetErrorString(ce));
            return ETD_OK;
        }
        launch_gemm_simt_f32((const float*)p->op[cur][0], (const float*)p->P[0], p->M, p->n, p->ninst * p->ncomp,
                             e, p->stream);
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(ETD_ERR_CUDA, "transform pass launch: %s", cudaGetErrorString(ce));
    return ETD_OK;
}

// d passes of config `slot` starting from operand buffer `cur`; the last pass
// uses final_mode and, if it writes an operand, splits it as final_split.
template <typename T>
etd_status run_chain(etd_plan* p, int& cur, int slot, int final_mode, int final_split, void* dst, int ld_dst,
                     long long bs_dst) {
    for (int pass = 0; pass < p->d; ++pass) {
        const bool last = pass == p->d - 1;
        etd_status s = run_pass<T>(p, cur, slot, last ? final_mode : EPI_SPLIT, last ? final_split : split_for(p, slot),
                                   dst, ld_dst, bs_dst);
        if (s != ETD_OK) return s;
        cur = 1 - cur;
    }
    return ETD_OK;
}

// Reaction (kind >= 0) or plain split (kind = -1) of a physical field into operand buffer 0.
template <typename T>
etd_status run_react(etd_plan* p, int kind, const void* in, int ld_in, long long bs_in, double t, int split) {
    Rx<T> r{};
    r.d = p->d;
    if (kind == ETD_RX_AC_FORCED) {
        const double lam = p->rp[0], pi = 3.14159265358979323846;
        r.decay = std::exp(-lam * t);
        r.psi_coef = -lam + p->d * pi * pi * p->kappa[0];
    }
    r.kind = kind;
    r.ncomp = p->ncomp;
    r.ninst = p->ninst;
    r.n = p->n;
    r.npts = p->npts;
    r.in = (const T*)in;
    r.ld_in = ld_in;
    r.bs_in = bs_in;
    r.out_hi = (T*)p->op[0][0];
    r.out_lo = (T*)p->op[0][1];
    r.out_lo2 = (T*)p->op[0][2];
    r.ld_out = p->ld;
    r.bs_out = p->bs;
    r.split = split;
    for (int i = 0; i < 4; ++i) r.rp[i] = (T)p->rp[i];
    TimerScope ts(p, 1);
    if constexpr (sizeof(T) == 8)
        launch_react_f64(r, p->stream);
    else
        launch_react_f32(r, p->stream);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(ETD_ERR_CUDA, "reaction launch: %s", cudaGetErrorString(ce));
    return ETD_OK;
}

// n_steps time steps. Every transform runs with config slot 0 except two, which
// run with p->out_slot (the accurate six-product kernel in TF32X3 mode): the
// U -> U^ transform that (re)builds the carried state, and the transform that
// produces the field handed back to the caller. Errors of the other transforms
// reach the state only through f(U) and f(W), scaled by tau.
// (Re)build the carried state U^ = T(U) when it is stale. The transform runs
// with the output slot: an error made here stays in the carried state.
template <typename T>
etd_status ensure_state(etd_plan* p, void* u) {
    if (p->uhat_valid && p->uhat_src == u) return ETD_OK;
    p->rx_ready = false;  // the rebuild below overwrites the operand buffers
    const int spo = split_for(p, p->out_slot);
    etd_status s = run_react<T>(p, -1, u, p->n, p->npts, p->t, spo);
    int cur = 0;
    if (s == ETD_OK) s = run_chain<T>(p, cur, p->out_slot, EPI_CARRY, spo, nullptr, 0, 0);
    if (s != ETD_OK) return s;
    p->uhat_valid = true;
    p->uhat_src = u;
    return ETD_OK;
}

// One time step from the carried state. Every transform runs with config slot 0
// except, when `last`, the one that produces the field handed back to the
// caller, which runs with p->out_slot (the accurate kernel of the split modes).
// Errors of the other transforms reach the state only through f(U) and f(W),
// scaled by tau.
// Reactions that act on each component at a point alone (rx_fusable) are
// evaluated in transform epilogues instead of the reaction kernel: f(t_{n+1}, W)
// (step a5) in the epilogue of the pass that produces W, and, when chain_rx,
// f(U+) of the next step (its a1) in the epilogue of the pass that returns U+;
// the next step then starts from those operand pieces.
template <typename T>
etd_status step_once(etd_plan* p, void* u, bool last, bool chain_rx) {
    const int n = p->n;
    const long long N = p->npts;
    const int sp0 = split_for(p, 0), spo = split_for(p, p->out_slot);
    const bool fuse = rx_fusable(p->reaction);
    etd_status s;
    int cur = 0;
    if (fuse && p->rx_ready && p->rx_src == u) {
        cur = p->rx_cur;  // f(t_n, U) pieces from the previous step's last epilogue
    } else if ((s = run_react<T>(p, p->reaction, u, n, N, p->t, sp0)) != ETD_OK) {
        return s;
    }
    p->rx_ready = false;
    if ((s = run_chain<T>(p, cur, 0, EPI_STAGE1, sp0, nullptr, 0, 0)) != ETD_OK) return s;
    if (fuse) {
        if ((s = run_chain<T>(p, cur, 0, EPI_REACT, sp0, nullptr, 0, 0)) != ETD_OK) return s;
    } else {
        if ((s = run_chain<T>(p, cur, 0, EPI_PLAIN, sp0, p->wphys, p->ld, p->bs)) != ETD_OK) return s;
        if ((s = run_react<T>(p, p->reaction, p->wphys, p->ld, p->bs, p->t + p->tau, sp0)) != ETD_OK) return s;
        cur = 0;
    }
    if ((s = run_chain<T>(p, cur, 0, EPI_STAGE2, last ? spo : sp0, nullptr, 0, 0)) != ETD_OK) return s;
    const bool chain = fuse && chain_rx;
    if ((s = run_chain<T>(p, cur, last ? p->out_slot : 0, chain ? EPI_PLAIN_REACT : EPI_PLAIN, sp0, u, n, N)) !=
        ETD_OK)
        return s;
    if (chain) {
        p->rx_ready = true;
        p->rx_cur = cur;
        p->rx_src = u;
    }
    p->t += p->tau;
    return ETD_OK;
}

// Step a8 on the device: FP64 max |u| and non-finite count of the field u (the
// plan's whole stacked field), then the bound check that raises ERR_DIVERGED.
// Asynchronous; etd_sync reports the outcome.
etd_status run_diag(etd_plan* p, const void* u) {
    const long long count = (long long)p->ninst * p->ncomp * p->npts;
    ETD_CUDA(cudaMemsetAsync(p->stats, 0, sizeof(double) * 2, p->stream));
    if (p->elem == 8)
        launch_stats_f64((const double*)u, count, p->stats, p->stream);
    else
        launch_stats_f32((const float*)u, count, p->stats, p->stream);
    launch_diag_check(p->stats, p->diag_max, (unsigned)p->steps_done, p->err, p->stats + 4, p->stream);
    ETD_CUDA(cudaGetLastError());
    return ETD_OK;
}

template <typename T>
etd_status step_impl(etd_plan* p, void* u, int n_steps) {
    etd_status s = ensure_state<T>(p, u);
    for (int it = 0; it < n_steps && s == ETD_OK; ++it) {
        s = step_once<T>(p, u, it == n_steps - 1, true);
        ++p->steps_done;
        if (s == ETD_OK && p->diag_every > 0 && p->steps_done % p->diag_every == 0) s = run_diag(p, u);
    }
    return s;
}

etd_status group_ensure_state(etd_plan* g, void* u) {
    return g->elem == 8 ? ensure_state<double>(g, u) : ensure_state<float>(g, u);
}

// Ensemble groups do not chain f(U+) across steps (a captured inner step must
// not depend on the step before it); f(W) is fused within each step.
etd_status group_step_once(etd_plan* g, void* u, bool last) {
    return g->elem == 8 ? step_once<double>(g, u, last, false) : step_once<float>(g, u, last, false);
}

// d E_l / dx of the factor family at x >= 0 (for the kappa gradients).
void factor_grid_derivs(int family, double x, double* de) {
    if (family == ETD_PADE_02 || family == ETD_PADE_04) {
        double D, dD, N[3], dN[3];
        if (family == ETD_PADE_02) {
            D = x * x + 2 * x + 2;
            dD = 2 * x + 2;
            N[0] = 2; N[1] = x + 2; N[2] = x + 1;
            dN[0] = 0; dN[1] = 1; dN[2] = 1;
        } else {
            D = (((x + 4) * x + 12) * x + 24) * x + 24;
            dD = ((4 * x + 12) * x + 24) * x + 24;
            N[0] = 24; N[1] = ((x + 4) * x + 12) * x + 24; N[2] = ((x + 3) * x + 8) * x + 12;
            dN[0] = 0; dN[1] = (3 * x + 8) * x + 12; dN[2] = (3 * x + 6) * x + 8;
        }
        for (int l = 0; l < 3; ++l) de[l] = (dN[l] * D - N[l] * dD) / (D * D);
        return;
    }
    // exact exponentials: E1 = e^{-x}, E2 = sum (-x)^j/(j+1)!, E3 = sum (-x)^j/(j+2)!
    de[0] = -std::exp(-x);
    if (x < 0.1) {
        double d2 = 0, d3 = 0, pw = 1.0, f2 = 2.0, f3 = 6.0;  // pw = (-1)^j x^{j-1}, j >= 1
        for (int j = 1; j < 14; ++j) {
            pw = (j == 1) ? -1.0 : pw * -x;
            d2 += j * pw / f2;
            d3 += j * pw / f3;
            f2 *= (j + 2);
            f3 *= (j + 3);
        }
        de[1] = d2;
        de[2] = d3;
    } else {
        const double e = std::exp(-x);
        de[1] = (e * (x + 1.0) - 1.0) / (x * x);
        de[2] = ((1.0 - e) * x - 2.0 * (x - 1.0 + e)) / (x * x * x);
    }
}

// out = T(in) (layouts of the caller, rows of n); kind >= 0 transforms f(in).
template <typename T>
etd_status xform(etd_plan* p, int kind, const void* in, void* out) {
    p->rx_ready = false;  // overwrites the operand buffers
    const int sp = split_for(p, p->out_slot);
    etd_status s = run_react<T>(p, kind, in, p->n, p->npts, p->t, sp);
    int cur = 0;
    if (s == ETD_OK) s = run_chain<T>(p, cur, p->out_slot, EPI_PLAIN, sp, out, p->n, p->npts);
    return s;
}

template <typename T>
etd_status spec(etd_plan* p, const void* in1, int x1, int s1, double a, const void* in2, int x2, int s2, double b,
                void* out) {
    SpecCombine<T> c{};
    c.ncomp = p->ncomp;
    c.d = p->d;
    c.n = p->n;
    c.npts = p->npts;
    c.grid = (const double*)p->grid;
    c.grid2 = (const float2*)p->grid2;
    c.in1 = (const T*)in1;
    c.xsel1 = x1;
    c.s1 = s1;
    c.alpha = a;
    c.in2 = (const T*)in2;
    c.xsel2 = x2;
    c.s2 = s2;
    c.beta = b;
    c.out = (T*)out;
    launch_spec_combine<T>(c, p->stream);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? ETD_OK : fail(ETD_ERR_CUDA, "adjoint kernel: %s", cudaGetErrorString(ce));
}

template <typename T>
etd_status vjp(etd_plan* p, const void* X, const void* V, const void* base, void* out) {
    ReactVjp<T> r{};
    r.kind = p->reaction;
    r.ncomp = p->ncomp;
    r.npts = p->npts;
    for (int i = 0; i < 4; ++i) r.rp[i] = p->rp[i];
    r.X = (const T*)X;
    r.V = (const T*)V;
    r.base = (const T*)base;
    r.out = (T*)out;
    launch_react_vjp<T>(r, p->stream);
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? ETD_OK : fail(ETD_ERR_CUDA, "adjoint kernel: %s", cudaGetErrorString(ce));
}

// One backward step from state U with lam = dL/dU^{n+1} on entry, dL/dU^n on exit.
template <typename T>
etd_status adjoint_step_impl(etd_plan* p, const void* U, void* lam) {
    void** w = p->adj_work;
    void *Fh = w[0], *Uh = w[1], *Wh = w[2], *W = w[3], *FWh = w[4], *Lh = w[5], *Gbh = w[6], *Gb = w[7];
    void *Wb = w[8], *Wbh = w[9], *Fbh = w[10], *Fb = w[11], *tmp = w[12], *tmpT = w[13];
    enum { X_ONE = 0, X_E1 = 1, X_E2 = 2, X_E3 = 3 };
    etd_status s = ETD_OK;
    // forward quantities of this step, in the eigenbasis
    if (s == ETD_OK) s = xform<T>(p, p->reaction, U, Fh);                            // F^ = T f(U)
    if (s == ETD_OK) s = xform<T>(p, -1, U, Uh);                                     // U^
    if (s == ETD_OK) s = spec<T>(p, Uh, X_E1, 1, 1.0, Fh, X_E2, 1, 1.0, Wh);         // W^
    if (s == ETD_OK) s = xform<T>(p, -1, Wh, W);                                     // W
    if (s == ETD_OK) s = xform<T>(p, p->reaction, W, FWh);                           // F_W^
    // backward
    if (s == ETD_OK) s = xform<T>(p, -1, lam, Lh);                                   // U+bar^
    if (s == ETD_OK) s = spec<T>(p, Lh, X_E3, 0, 1.0, nullptr, 0, 0, 0.0, Gbh);      // Gbar^ = tau E3 U+bar^
    if (s == ETD_OK) s = xform<T>(p, -1, Gbh, Gb);                                   // Gbar
    if (s == ETD_OK) s = vjp<T>(p, W, Gb, lam, Wb);                                  // Wbar
    if (s == ETD_OK) s = xform<T>(p, -1, Wb, Wbh);                                   // Wbar^
    if (s == ETD_OK) s = spec<T>(p, Wbh, X_E2, 1, 1.0, Gbh, X_ONE, 1, -1.0, Fbh);    // Fbar^
    if (s == ETD_OK) s = xform<T>(p, -1, Fbh, Fb);                                   // Fbar
    if (s == ETD_OK) s = spec<T>(p, Wbh, X_E1, 1, 1.0, nullptr, 0, 0, 0.0, tmp);     // X1 S Wbar^
    if (s == ETD_OK) s = xform<T>(p, -1, tmp, tmpT);
    if (s != ETD_OK) return s;
    GradKappa<T> gk{};
    gk.ncomp = p->ncomp;
    gk.d = p->d;
    gk.n = p->n;
    gk.npts = p->npts;
    gk.grid = (const double*)p->grid;
    gk.dgrid = p->adj_dgrid;
    gk.grid2 = (const float2*)p->grid2;
    gk.dgrid2 = p->adj_dgrid2;
    gk.Lh = (const T*)Lh;
    gk.Gbh = (const T*)Gbh;
    gk.Wbh = (const T*)Wbh;
    gk.Uh = (const T*)Uh;
    gk.Fh = (const T*)Fh;
    gk.FWh = (const T*)FWh;
    gk.out = p->adj_acc;
    launch_grad_kappa<T>(gk, p->stream);
    GradRx<T> gr{};
    gr.kind = p->reaction;
    gr.ncomp = p->ncomp;
    gr.npts = p->npts;
    for (int i = 0; i < 4; ++i) gr.rp[i] = p->rp[i];
    gr.U = (const T*)U;
    gr.W = (const T*)W;
    gr.Gb = (const T*)Gb;
    gr.Fb = (const T*)Fb;
    gr.out = p->adj_acc + 2;
    launch_grad_rx<T>(gr, p->stream);
    return vjp<T>(p, U, Fb, tmpT, lam);  // Ubar = X1 S Wbar + J_f(U)^T Fbar
}

template <typename T>
etd_status adjoint_impl(etd_plan* p, const void* u_ckpt, void* lam, int n_steps) {
    const size_t fbytes = (size_t)p->ncomp * p->npts * p->elem;
    while ((int)p->adj_traj.size() < n_steps) {
        void* f = nullptr;
        etd_status s = dalloc(p, &f, fbytes);
        if (s != ETD_OK) return s;
        p->adj_traj.push_back(f);
    }
    // forward states U^0 .. U^{N-1} of the window, recomputed from the checkpoint
    // in one work field (its carried spectral state stays valid from step to
    // step, as in the forward run) and copied out after every step
    const double t0 = p->t;
    void* work = p->adj_work[12];  // free until the backward steps
    ETD_CUDA(cudaMemcpyAsync(p->adj_traj[0], u_ckpt, fbytes, cudaMemcpyDeviceToDevice, p->stream));
    if (n_steps > 1) ETD_CUDA(cudaMemcpyAsync(work, u_ckpt, fbytes, cudaMemcpyDeviceToDevice, p->stream));
    for (int j = 1; j < n_steps; ++j) {
        etd_status s = step_impl<T>(p, work, 1);
        if (s != ETD_OK) return s;
        ETD_CUDA(cudaMemcpyAsync(p->adj_traj[j], work, fbytes, cudaMemcpyDeviceToDevice, p->stream));
    }
    p->t = t0;
    p->uhat_valid = false;  // the carried state now belongs to the recomputed window
    for (int j = n_steps - 1; j >= 0; --j) {
        etd_status s = adjoint_step_impl<T>(p, p->adj_traj[j], lam);
        if (s != ETD_OK) return s;
    }
    return ETD_OK;
}

etd_status check_device_ptr(const void* ptr, const char* what) {
    if (!ptr) return fail(ETD_ERR_INVALID_ARG, "%s is NULL", what);
    if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return fail(ETD_ERR_INVALID_ARG, "%s is not 16-byte aligned", what);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ETD_ERR_INVALID_ARG, "%s: %s", what, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(ETD_ERR_INVALID_ARG, "%s is not device memory", what);
    return ETD_OK;
}

}  // namespace

namespace etd {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace etd

extern "C" {

etd_status etd_options_default(etd_options* opt) {
    if (!opt) return fail(ETD_ERR_INVALID_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = ETD_PREC_FP64_SPLIT;
    opt->reaction = ETD_RX_ALLEN_CAHN;
    opt->n_comp = 1;
    return ETD_OK;
}

}  // extern "C"

namespace {

etd_status validate_options(int d, int m, int pade_order, const etd_options& opt) {
    if (d != 2 && d != 3) return fail(ETD_ERR_INVALID_ARG, "d must be 2 or 3 (got %d)", d);
    const int mmax = (d == 2) ? 16384 : 1024;
    if (m < 2 || m > mmax) return fail(ETD_ERR_INVALID_ARG, "m must be in [2, %d] (got %d)", mmax, m);
    if (pade_order != ETD_PADE_02 && pade_order != ETD_PADE_04 && pade_order != ETD_EXACT_EXP)
        return fail(ETD_ERR_INVALID_ARG, "pade_order must be 2, 4 or 0 (exact exponential)");
    if (opt.n_comp < 1 || opt.n_comp > 2) return fail(ETD_ERR_INVALID_ARG, "n_comp must be 1 or 2");
    if (opt.flags & ~ETD_FLAG_AUTOTUNE) return fail(ETD_ERR_INVALID_ARG, "unknown bits in flags (0x%x)", opt.flags);
    if (opt.diag_every < 0) return fail(ETD_ERR_INVALID_ARG, "diag_every must be >= 0");
    if (std::isnan(opt.diag_max_abs)) return fail(ETD_ERR_INVALID_ARG, "diag_max_abs is NaN");
    if (opt.reaction < ETD_RX_NONE || opt.reaction > ETD_RX_AC_FORCED)
        return fail(ETD_ERR_INVALID_ARG, "unknown reaction");
    if (opt.reaction == ETD_RX_FHN && opt.n_comp != 2)
        return fail(ETD_ERR_INVALID_ARG, "FitzHugh-Nagumo needs n_comp = 2");
    if ((opt.reaction == ETD_RX_ALLEN_CAHN || opt.reaction == ETD_RX_SINGULAR || opt.reaction == ETD_RX_AC_FORCED) &&
        opt.n_comp != 1)
        return fail(ETD_ERR_INVALID_ARG, "this reaction needs n_comp = 1");
    if (opt.precision == ETD_PREC_DST32) {
        const int N = m + 1;
        if (N < 16 || N > 8192 || (N & (N - 1)))
            return fail(ETD_ERR_UNSUPPORTED, "ETD_PREC_DST32 needs m + 1 a power of two in [16, 8192] (m = %d)", m);
    }
    if ((opt.precision == ETD_PREC_FP64_SPLIT || opt.precision == ETD_PREC_FP64_SPLIT40 ||
         opt.precision == ETD_PREC_FP64_SPLIT32) &&
        m > OZ_MAX_N)  // the 2D limit; exact int32 level sums up to it
        return fail(ETD_ERR_UNSUPPORTED, "the FP64-split precisions need m <= %d (exact level sums; m = %d)", OZ_MAX_N,
                    m);
    if (opt.precision < ETD_PREC_FP64 || opt.precision > ETD_PREC_FP64_SPLIT32)
        return fail(ETD_ERR_INVALID_ARG, "unknown precision");
    return ETD_OK;
}

etd_status validate_scalars(double kappa, double q, double dt) {
    if (!(kappa > 0) || !std::isfinite(kappa)) return fail(ETD_ERR_INVALID_ARG, "kappa must be > 0");
    if (!(q >= 0) || !std::isfinite(q)) return fail(ETD_ERR_INVALID_ARG, "q must be >= 0");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(ETD_ERR_INVALID_ARG, "dt must be > 0");
    return ETD_OK;
}

// ---- autotuner (ETD_FLAG_AUTOTUNE) ----
// Key: (M, n, nbatch, products, bf16, accurate); value: the chosen configuration.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, TcConfig> g_tune_cache;

// Time the candidate configurations of config slot `slot` on the plan's own
// operand buffers (a split pass from buffer 0 into buffer 1: the buffers hold
// zeros at this point, and nothing in them is needed afterwards) and keep the
// fastest in p->tc[slot].
etd_status autotune_slot(etd_plan* p, int slot) {
    const TcConfig& cur = p->tc[slot];
    const auto key = std::make_tuple(p->M, p->n, p->ninst * p->ncomp, cur.products, cur.bf16 ? 1 : 0,
                                     cur.accurate ? 1 : 0);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->tc[slot] = it->second;
            return ETD_OK;
        }
    }
    const int nb = p->ninst * p->ncomp;
    TcConfig cand[4];
    const int nc = tc_candidates(p->M, p->n, cur.products, nb, cur.bf16, cur.accurate, cand, 4);
    int best = 0;
    if (nc > 1) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ETD_CUDA(cudaEventCreate(&e0));
        ETD_CUDA(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        etd_status st = ETD_OK;
        for (int i = 0; i < nc && st == ETD_OK; ++i) {
            const void* a[2][3];
            for (int x = 0; x < 2; ++x)
                for (int y = 0; y < 3; ++y) a[x][y] = p->op[x][y];
            const void* pp[3] = {p->P[0], p->P[1], p->P[2]};
            const int bn_slot[2] = {cand[i].bn, cand[i].bn};
            TcMaps* maps = nullptr;
            cudaError_t ce = tc_maps_create(&maps, p->M, p->n, nb, p->ld, a, 2, pp, bn_slot, p->bf16);
            if (ce != cudaSuccess) {
                st = fail(ETD_ERR_CUDA, "autotune tensor maps: %s %s", cudaGetErrorString(ce), tc_last_driver_error());
                break;
            }
            Epi<float> e = base_epi<float>(p);
            e.mode = EPI_SPLIT;
            e.split = split_for(p, slot);
            e.op_hi = (float*)p->op[1][0];
            e.op_lo = (float*)p->op[1][1];
            e.op_lo2 = (float*)p->op[1][2];
            const int reps = 3;
            ce = launch_gemm_tc(cand[i], slot, maps, 0, p->M, p->n, nb, e, p->err, p->stream);  // warm-up
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, p->stream);
            for (int r = 0; r < reps && ce == cudaSuccess; ++r)
                ce = launch_gemm_tc(cand[i], slot, maps, 0, p->M, p->n, nb, e, p->err, p->stream);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, p->stream);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
            tc_maps_destroy(maps);
            unsigned flags = 0;
            if (ce == cudaSuccess) ce = cudaMemcpy(&flags, p->err, sizeof flags, cudaMemcpyDeviceToHost);
            if (ce != cudaSuccess) {
                st = fail(ETD_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(ce));
            } else if (flags) {
                st = fail(flags & ERR_TIMEOUT ? ETD_ERR_TIMEOUT : ETD_ERR_CUDA, "autotune: device error flags 0x%x",
                          flags);
            } else if (ms < best_ms) {
                best_ms = ms;
                best = i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != ETD_OK) return st;
    }
    p->tc[slot] = cand[best];
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = cand[best];
    return ETD_OK;
}

// A plan for ninst instances on the same grid (d, n): kap[i * ncomp + c] is the
// diffusivity of component c of instance i, qv[i] and dtv[i] its potential and
// time step. Every (instance, component) gets its own factor grids; P is shared.
etd_status build_plan(etd_plan** out, int d, int m, int ninst, const double* kap, const double* qv, const double* dtv,
                      int pade_order, const etd_options& opt) {
    *out = nullptr;
    etd_plan* p = new (std::nothrow) etd_plan();
    if (!p) return fail(ETD_ERR_OOM, "host allocation failed");
    p->d = d;
    p->n = m;
    p->ninst = ninst;
    p->ncomp = opt.n_comp;
    p->precision = opt.precision;
    p->pade = pade_order;
    p->reaction = opt.reaction;
    std::memcpy(p->rp, opt.rx_params, sizeof p->rp);
    for (int c = 0; c < p->ncomp; ++c) p->kappa[c] = kap[c];
    p->q = qv[0];
    p->tau = dtv[0];
    p->stream = (cudaStream_t)opt.stream;
    p->diag_every = opt.diag_every;
    p->diag_max = opt.diag_max_abs;
    p->oz_s = opt.precision == ETD_PREC_FP64_SPLIT     ? 6
              : opt.precision == ETD_PREC_FP64_SPLIT40 ? 5
              : opt.precision == ETD_PREC_FP64_SPLIT32 ? 4
                                                       : 0;
    p->ozaki = p->oz_s > 0;
    p->elem = (opt.precision == ETD_PREC_FP64 || p->ozaki) ? 8 : 4;
    p->bf16 = (opt.precision == ETD_PREC_BF16X3 || opt.precision == ETD_PREC_BF16X6);
    p->use_tc = p->bf16 || opt.precision == ETD_PREC_TF32 || opt.precision == ETD_PREC_TF32X3 ||
                opt.precision == ETD_PREC_TF32X6;
    p->op_elem = p->bf16 ? 2 : p->elem;
    p->dst = opt.precision == ETD_PREC_DST32;
    const int n = m;
    const int nb = ninst * p->ncomp;
    p->M = (d == 2) ? n : n * n;
    p->mq = (d == 2) ? 1 : n;
    p->ld = (n + 7) / 8 * 8;  // rows start on 16-byte boundaries for 2- and 4-byte values
    p->bs = (long long)p->M * p->ld;
    p->npts = (long long)p->M * n;

    // ---- FP64 precompute ----
    const double h = 1.0 / (n + 1);
    const double pi = 3.14159265358979323846;
    std::vector<double> P((size_t)n * n);
    const double scale = std::sqrt(2.0 / (n + 1));
    const long long period = 2LL * (n + 1);
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < n; ++k) {
            const long long r = ((long long)(j + 1) * (k + 1)) % period;  // reduce before sin()
            P[(size_t)j * n + k] = scale * std::sin(pi * (double)r / (double)(n + 1));
        }
    std::vector<double> grid((size_t)nb * 3 * n);
    for (int b = 0; b < nb; ++b) {
        const int inst = b / p->ncomp;
        const double dt = dtv[inst], q = qv[inst];
        for (int k = 0; k < n; ++k) {
            const double sk = std::sin(pi * (k + 1) / (2.0 * (n + 1)));
            const double lam = 4.0 * kap[b] / (h * h) * sk * sk + q / d;
            double e[3];
            factor_grids(pade_order, dt * lam, e);
            grid[((size_t)b * 3 + 0) * n + k] = e[0];
            grid[((size_t)b * 3 + 1) * n + k] = dt * e[1];
            grid[((size_t)b * 3 + 2) * n + k] = dt * e[2];
        }
    }

    // ---- tensor-core configurations ----
    if (p->use_tc) {
        const int prod0 = opt.precision == ETD_PREC_TF32
                              ? 1
                              : ((opt.precision == ETD_PREC_TF32X6 || opt.precision == ETD_PREC_BF16X6) ? 6 : 3);
        // slot 0: every per-step pass; slot 1: the transforms whose error stays in
        // the result (state rebuild, returned field), the ACCURATE six-product kernel.
        // The six-product modes run every pass ACCURATE: with all six products in
        // one k-block accumulator a pass is about as slow and no more accurate than
        // the three-product split (the tensor cores' truncating accumulation, not
        // the dropped lo*lo term, sets the error).
        p->tc[0] = tc_choose(p->M, n, prod0, nb, p->bf16, prod0 == 6);
        if (prod0 > 1) {
            p->tc[1] = tc_choose(p->M, n, 6, nb, p->bf16, true);
            p->out_slot = 1;
        } else {
            p->tc[1] = p->tc[0];
        }
        p->pieces = p->tc[0].pieces > p->tc[1].pieces ? p->tc[0].pieces : p->tc[1].pieces;
    }

    // ---- device buffers ----
    etd_status s = ETD_OK;
    const size_t E = p->elem;
    const size_t field_bytes = (size_t)nb * p->bs * E;
    const size_t state_bytes = (size_t)nb * p->bs * sizeof(double);
    const size_t pbytes = (size_t)n * p->ld * p->op_elem;
    const size_t op_bytes = (size_t)nb * p->bs * p->op_elem;
    // the sine-transform path needs no P: its twiddles and a scratch field instead
    for (int j = 0; j < (p->dst || p->ozaki ? 0 : p->pieces) && s == ETD_OK; ++j) s = dalloc(p, &p->P[j], pbytes);
    // FP64-split: the operand's slice planes, P's slice planes, the scale words
    for (int i = 0; i < (p->ozaki ? p->oz_s : 0) && s == ETD_OK; ++i) {
        s = dalloc(p, &p->oz_slices[i], oz_plane_bytes((long long)nb * p->M, n, OZ_TILE_ROWS_A));
        if (s == ETD_OK) s = dalloc(p, &p->oz_P[i], oz_plane_bytes(n, n, OZ_TILE_ROWS_P));
    }
    if (s == ETD_OK && p->ozaki) s = dalloc(p, (void**)&p->oz_rexp, sizeof(int) * (size_t)nb * p->M);
    if (s == ETD_OK && p->dst) s = dalloc(p, (void**)&p->dst_tw, sizeof(float2) * (size_t)(2 * (n + 1) - 1));
    if (s == ETD_OK && p->dst) s = dalloc(p, &p->dst_tmp, field_bytes);
    if (s == ETD_OK) s = dalloc(p, &p->grid, (size_t)nb * 3 * n * sizeof(double));
    if (s == ETD_OK) s = dalloc(p, &p->grid2, (size_t)nb * 3 * n * 2 * sizeof(float));
    if (s == ETD_OK) s = dalloc(p, &p->uhat, state_bytes);
    if (s == ETD_OK) s = dalloc(p, &p->zhat, state_bytes);
    if (s == ETD_OK) s = dalloc(p, &p->wphys, field_bytes);
    for (int i = 0; i < 2 && s == ETD_OK; ++i)
        for (int j = 0; j < p->pieces && s == ETD_OK; ++j) s = dalloc(p, &p->op[i][j], op_bytes);
    if (s == ETD_OK) s = dalloc(p, (void**)&p->err, sizeof(unsigned) * 4);
    if (s == ETD_OK) s = dalloc(p, (void**)&p->stats, sizeof(double) * 8);
    if (s != ETD_OK) {
        free_plan(p);
        return s;
    }
    // P in its pieces: FP64 for ETD_PREC_FP64, FP32 for FP32 products, TF32
    // pieces (each rounded from the FP64 remainder) for the tensor-core modes
    cudaError_t ce = cudaSuccess;
    if (p->dst) {  // FFT twiddles by stage: half - 1 + pos -> e^{-i pi pos / half}, half = 1, 2, .., N/2
        const int N = 2 * (n + 1);
        std::vector<float2> tw((size_t)(N - 1));
        const double pi = 3.14159265358979323846;
        for (int half = 1; half < N; half *= 2)
            for (int pos = 0; pos < half; ++pos) {
                const double a = -pi * pos / half;
                tw[(size_t)(half - 1 + pos)] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        ce = cudaMemcpy(p->dst_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
    }
    if (p->ozaki && ce == cudaSuccess) {
        // tiled planes: their padding (rows past the last, values past n) stays zero
        const size_t pplane = oz_plane_bytes(n, n, OZ_TILE_ROWS_P) / 2;
        std::vector<uint16_t> planes((size_t)p->oz_s * pplane, 0);
        uint16_t* ptrs[OZ_S] = {nullptr};
        for (int i = 0; i < p->oz_s; ++i) ptrs[i] = planes.data() + (size_t)i * pplane;
        p->oz_pexp = oz_slice_host(P.data(), n, p->oz_s, ptrs);
        for (int i = 0; i < p->oz_s && ce == cudaSuccess; ++i)
            ce = cudaMemcpy(p->oz_P[i], ptrs[i], pplane * 2, cudaMemcpyHostToDevice);
        for (int i = 0; i < p->oz_s && ce == cudaSuccess; ++i)
            ce = cudaMemset(p->oz_slices[i], 0, oz_plane_bytes((long long)nb * p->M, n, OZ_TILE_ROWS_A));
        if (ce == cudaSuccess) ce = oz_prepare();
    }
    for (int j = 0; j < (p->dst || p->ozaki ? 0 : p->pieces) && ce == cudaSuccess; ++j) {
        std::vector<char> hostbuf(pbytes, 0);
        for (int r = 0; r < n; ++r)
            for (int k = 0; k < n; ++k) {
                double v = P[(size_t)r * n + k];
                const size_t o = (size_t)r * p->ld + k;
                if (E == 8) {
                    ((double*)hostbuf.data())[o] = v;
                } else if (!p->use_tc) {
                    ((float*)hostbuf.data())[o] = (float)v;
                } else if (p->bf16) {
                    uint16_t piece = 0;
                    for (int q = 0; q <= j; ++q) {
                        piece = bf16_round_host((float)v);
                        v -= (double)bf16_to_float_host(piece);
                    }
                    ((uint16_t*)hostbuf.data())[o] = piece;
                } else {
                    float piece = 0.f;
                    for (int q = 0; q <= j; ++q) {
                        piece = tf32_round_host((float)v);
                        v -= (double)piece;
                    }
                    ((float*)hostbuf.data())[o] = piece;
                }
            }
        ce = cudaMemcpy(p->P[j], hostbuf.data(), pbytes, cudaMemcpyHostToDevice);
    }
    if (ce == cudaSuccess) ce = cudaMemcpy(p->grid, grid.data(), grid.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) {  // double-float copy: hi = rn(g), lo = rn(g - hi)
        std::vector<float> g2(grid.size() * 2);
        for (size_t i = 0; i < grid.size(); ++i) {
            g2[2 * i] = (float)grid[i];
            g2[2 * i + 1] = (float)(grid[i] - (double)g2[2 * i]);
        }
        ce = cudaMemcpy(p->grid2, g2.data(), g2.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    // zero the padded operand columns once (they are never written by the passes)
    for (int i = 0; i < 2 && ce == cudaSuccess; ++i)
        for (int j = 0; j < p->pieces && ce == cudaSuccess; ++j) ce = cudaMemset(p->op[i][j], 0, op_bytes);
    if (ce == cudaSuccess) ce = cudaMemset(p->err, 0, sizeof(unsigned) * 4);
    if (ce != cudaSuccess) {
        free_plan(p);
        return fail(ETD_ERR_CUDA, "plan upload: %s", cudaGetErrorString(ce));
    }
    if (p->use_tc && (opt.flags & ETD_FLAG_AUTOTUNE)) {
        etd_status st = autotune_slot(p, 0);
        if (st == ETD_OK && p->out_slot != 0) st = autotune_slot(p, p->out_slot);
        if (st != ETD_OK) {
            free_plan(p);
            return st;
        }
    }
    if (p->use_tc) {
        const void* a[2][3];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) a[i][j] = p->op[i][j];
        const void* pp[3] = {p->P[0], p->P[1], p->P[2]};
        const int bn_slot[2] = {p->tc[0].bn, p->tc[1].bn};
        ce = tc_maps_create(&p->maps, p->M, n, nb, p->ld, a, 2, pp, bn_slot, p->bf16);
        if (ce != cudaSuccess) {
            std::string why = tc_last_driver_error();
            free_plan(p);
            return fail(ETD_ERR_CUDA, "tensor maps: %s %s", cudaGetErrorString(ce), why.c_str());
        }
    }
    *out = p;
    return ETD_OK;
}

}  // namespace

extern "C" {

etd_status etd_plan_create(etd_plan** out, int d, int m, double kappa, double q, double dt, int pade_order,
                           const etd_options* opt_in) {
    if (!out) return fail(ETD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    etd_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        etd_options_default(&opt);
    etd_status s = validate_options(d, m, pade_order, opt);
    if (s == ETD_OK) s = validate_scalars(kappa, q, dt);
    if (s != ETD_OK) return s;
    double kap[2];
    for (int c = 0; c < opt.n_comp; ++c) kap[c] = (opt.kappa_comp[c] > 0) ? opt.kappa_comp[c] : kappa;
    return build_plan(out, d, m, 1, kap, &q, &dt, pade_order, opt);
}

etd_status etd_batch_create(etd_plan** out, int count, const int* d, const int* m, const double* kappa,
                            const double* q, const double* dt, int pade_order, const etd_options* opt_in) {
    if (!out) return fail(ETD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !d || !m || !kappa || !q || !dt) return fail(ETD_ERR_INVALID_ARG, "empty or NULL instance arrays");
    etd_options opt;
    if (opt_in)
        opt = *opt_in;
    else
        etd_options_default(&opt);
    if (opt.reaction == ETD_RX_AC_FORCED)
        return fail(ETD_ERR_INVALID_ARG, "time-dependent reactions are not supported in a batch");
    for (int i = 0; i < count; ++i) {
        etd_status s = validate_options(d[i], m[i], pade_order, opt);
        if (s == ETD_OK) s = validate_scalars(kappa[i], q[i], dt[i]);
        if (s != ETD_OK) return s;
    }
    etd_plan* B = new (std::nothrow) etd_plan();
    if (!B) return fail(ETD_ERR_OOM, "host allocation failed");
    B->is_batch = true;
    B->count = count;
    B->ncomp = opt.n_comp;
    B->precision = opt.precision;
    B->elem = (opt.precision == ETD_PREC_FP64 || opt.precision == ETD_PREC_FP64_SPLIT ||
               opt.precision == ETD_PREC_FP64_SPLIT40 || opt.precision == ETD_PREC_FP64_SPLIT32)
                  ? 8
                  : 4;
    B->stream = (cudaStream_t)opt.stream;
    // group the instances by grid (d, n), in order of first appearance
    std::vector<std::pair<int, int>> keys;
    for (int i = 0; i < count; ++i) {
        size_t gi = 0;
        while (gi < keys.size() && keys[gi] != std::make_pair(d[i], m[i])) ++gi;
        if (gi == keys.size()) {
            keys.push_back({d[i], m[i]});
            B->members.emplace_back();
        }
        B->members[gi].push_back(i);
    }
    etd_status s = ETD_OK;
    cudaError_t ce = cudaEventCreateWithFlags(&B->ev_start, cudaEventDisableTiming);
    for (size_t gi = 0; gi < keys.size() && s == ETD_OK && ce == cudaSuccess; ++gi) {
        const std::vector<int>& mem = B->members[gi];
        const int ni = (int)mem.size();
        std::vector<double> kap((size_t)ni * opt.n_comp), qv(ni), dtv(ni);
        for (int li = 0; li < ni; ++li) {
            const int i = mem[li];
            for (int c = 0; c < opt.n_comp; ++c)
                kap[(size_t)li * opt.n_comp + c] = (c > 0 && opt.kappa_comp[c] > 0) ? opt.kappa_comp[c] : kappa[i];
            qv[li] = q[i];
            dtv[li] = dt[i];
        }
        etd_options gopt = opt;
        cudaStream_t gs = nullptr;
        ce = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
        if (ce != cudaSuccess) break;
        gopt.stream = gs;
        etd_plan* g = nullptr;
        s = build_plan(&g, keys[gi].first, keys[gi].second, ni, kap.data(), qv.data(), dtv.data(), pade_order, gopt);
        if (s != ETD_OK) {
            cudaStreamDestroy(gs);
            break;
        }
        B->groups.push_back(g);
        void* f = nullptr;
        s = dalloc(B, &f, (size_t)ni * opt.n_comp * g->npts * g->elem);
        B->gfield.push_back(f);
        cudaEvent_t ev = nullptr;
        if (s == ETD_OK) ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        B->ev_done.push_back(ev);
    }
    if (s == ETD_OK && ce != cudaSuccess) s = fail(ETD_ERR_CUDA, "batch streams/events: %s", cudaGetErrorString(ce));
    if (s != ETD_OK) {
        free_plan(B);
        return s;
    }
    for (etd_plan* g : B->groups) B->workspace += g->workspace;
    *out = B;
    return ETD_OK;
}

etd_status etd_batch_step(etd_plan* B, void* const* u_dev, int n_steps) {
    if (!B || !B->is_batch) return fail(ETD_ERR_INVALID_ARG, "not a batch plan (use etd_batch_create)");
    if (!u_dev) return fail(ETD_ERR_INVALID_ARG, "u_dev is NULL");
    if (n_steps < 0) return fail(ETD_ERR_INVALID_ARG, "n_steps must be >= 0");
    for (long long i = 0; i < B->count; ++i) {
        etd_status s = check_device_ptr(u_dev[i], "u_dev[i]");
        if (s != ETD_OK) return s;
    }
    if (n_steps == 0) return ETD_OK;
    // the carried spectral states stay valid only for the same fields as last time
    bool same = B->last_ptrs.size() == (size_t)B->count;
    for (long long i = 0; same && i < B->count; ++i) same = B->last_ptrs[i] == u_dev[i];
    if (!same) {
        for (etd_plan* g : B->groups) g->uhat_valid = false;
        B->last_ptrs.assign(u_dev, u_dev + B->count);
    }
    const size_t G = B->groups.size();
    // gather every instance's field into its group's buffer, (re)build stale states
    ETD_CUDA(cudaEventRecord(B->ev_start, B->stream));
    for (size_t gi = 0; gi < G; ++gi) {
        etd_plan* g = B->groups[gi];
        const size_t inst_bytes = (size_t)g->ncomp * g->npts * g->elem;
        char* gf = static_cast<char*>(B->gfield[gi]);
        ETD_CUDA(cudaStreamWaitEvent(g->stream, B->ev_start, 0));
        for (size_t li = 0; li < B->members[gi].size(); ++li)
            ETD_CUDA(cudaMemcpyAsync(gf + li * inst_bytes, u_dev[B->members[gi][li]], inst_bytes,
                                     cudaMemcpyDeviceToDevice, g->stream));
        etd_status s = group_ensure_state(g, gf);
        if (s != ETD_OK) return s;
        ETD_CUDA(cudaEventRecord(B->ev_done[gi], g->stream));
        ETD_CUDA(cudaStreamWaitEvent(B->stream, B->ev_done[gi], 0));
    }
    // inner steps: one CUDA graph of all groups' launches (forked over the group
    // streams), captured once and replayed; without timing events only, since
    // those are recorded per launch by the host
    const bool use_graph = n_steps > 1 && !B->timing;
    if (use_graph && !B->step_graph) {
        cudaGraph_t graph = nullptr;
        if (!B->cap_stream) ETD_CUDA(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
        ETD_CUDA(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
        etd_status s = ETD_OK;
        cudaError_t ce = cudaEventRecord(B->ev_start, B->cap_stream);
        for (size_t gi = 0; gi < G && s == ETD_OK && ce == cudaSuccess; ++gi) {
            etd_plan* g = B->groups[gi];
            ce = cudaStreamWaitEvent(g->stream, B->ev_start, 0);
            const double t0 = g->t;
            if (ce == cudaSuccess) s = group_step_once(g, B->gfield[gi], false);
            g->t = t0;  // the replays advance time below
            if (ce == cudaSuccess) ce = cudaEventRecord(B->ev_done[gi], g->stream);
            if (ce == cudaSuccess) ce = cudaStreamWaitEvent(B->cap_stream, B->ev_done[gi], 0);
        }
        cudaError_t ce2 = cudaStreamEndCapture(B->cap_stream, &graph);
        if (s != ETD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (ce == cudaSuccess) ce = ce2;
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&B->step_graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            B->step_graph = nullptr;
            return fail(ETD_ERR_CUDA, "capturing the ensemble step: %s", cudaGetErrorString(ce));
        }
    }
    for (int it = 0; it < n_steps - 1; ++it) {
        if (use_graph) {
            ETD_CUDA(cudaGraphLaunch(B->step_graph, B->stream));
            for (etd_plan* g : B->groups) g->t += g->tau;
        } else {
            ETD_CUDA(cudaEventRecord(B->ev_start, B->stream));
            for (size_t gi = 0; gi < G; ++gi) {
                etd_plan* g = B->groups[gi];
                ETD_CUDA(cudaStreamWaitEvent(g->stream, B->ev_start, 0));
                etd_status s = group_step_once(g, B->gfield[gi], false);
                if (s != ETD_OK) return s;
                ETD_CUDA(cudaEventRecord(B->ev_done[gi], g->stream));
                ETD_CUDA(cudaStreamWaitEvent(B->stream, B->ev_done[gi], 0));
            }
        }
    }
    // last step (accurate output transform) and scatter back
    ETD_CUDA(cudaEventRecord(B->ev_start, B->stream));
    for (size_t gi = 0; gi < G; ++gi) {
        etd_plan* g = B->groups[gi];
        const size_t inst_bytes = (size_t)g->ncomp * g->npts * g->elem;
        char* gf = static_cast<char*>(B->gfield[gi]);
        ETD_CUDA(cudaStreamWaitEvent(g->stream, B->ev_start, 0));
        etd_status s = group_step_once(g, gf, true);
        if (s == ETD_OK && g->diag_every > 0) {
            g->steps_done += n_steps;
            s = run_diag(g, gf);
        }
        if (s != ETD_OK) return s;
        for (size_t li = 0; li < B->members[gi].size(); ++li)
            ETD_CUDA(cudaMemcpyAsync(u_dev[B->members[gi][li]], gf + li * inst_bytes, inst_bytes,
                                     cudaMemcpyDeviceToDevice, g->stream));
        ETD_CUDA(cudaEventRecord(B->ev_done[gi], g->stream));
        ETD_CUDA(cudaStreamWaitEvent(B->stream, B->ev_done[gi], 0));
    }
    return ETD_OK;
}

etd_status etd_step(etd_plan* p, void* u_dev, int n_steps) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    if (p->is_batch) return fail(ETD_ERR_INVALID_ARG, "a batch plan is stepped with etd_batch_step");
    if (n_steps < 0) return fail(ETD_ERR_INVALID_ARG, "n_steps must be >= 0");
    etd_status s = check_device_ptr(u_dev, "u_dev");
    if (s != ETD_OK) return s;
    if (n_steps == 0) return ETD_OK;
    return (p->elem == 8) ? step_impl<double>(p, u_dev, n_steps) : step_impl<float>(p, u_dev, n_steps);
}

etd_status etd_step_adjoint(etd_plan* p, const void* u_ckpt, void* lambda_dev, int n_steps, double* grad_kappa,
                            double* grad_rx) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    if (p->is_batch) return fail(ETD_ERR_INVALID_ARG, "the adjoint works on single plans");
    if (n_steps < 1) return fail(ETD_ERR_INVALID_ARG, "n_steps must be >= 1");
    if (p->reaction == ETD_RX_AC_FORCED)
        return fail(ETD_ERR_UNSUPPORTED, "the adjoint supports autonomous reactions only");
    etd_status s = check_device_ptr(u_ckpt, "u_ckpt");
    if (s == ETD_OK) s = check_device_ptr(lambda_dev, "lambda_dev");
    if (s != ETD_OK) return s;
    const size_t fbytes = (size_t)p->ncomp * p->npts * p->elem;
    if (!p->adj_acc) {
        for (int i = 0; i < 14 && s == ETD_OK; ++i) s = dalloc(p, &p->adj_work[i], fbytes);
        if (s == ETD_OK) s = dalloc(p, (void**)&p->adj_acc, 8 * sizeof(double));
        if (s == ETD_OK) s = dalloc(p, (void**)&p->adj_dgrid, (size_t)p->ncomp * 3 * p->n * sizeof(double));
        if (s == ETD_OK) s = dalloc(p, (void**)&p->adj_dgrid2, (size_t)p->ncomp * 3 * p->n * sizeof(float2));
        if (s != ETD_OK) return s;
        // d/dkappa of E1(tau lambda), tau E2, tau E3: tau mu E_l'(tau lambda), mu = dlambda/dkappa
        const int n = p->n;
        const double h = 1.0 / (n + 1), pi = 3.14159265358979323846;
        std::vector<double> dg((size_t)p->ncomp * 3 * n);
        for (int c = 0; c < p->ncomp; ++c)
            for (int k = 0; k < n; ++k) {
                const double sk = std::sin(pi * (k + 1) / (2.0 * (n + 1)));
                const double mu = 4.0 / (h * h) * sk * sk;
                const double lam = p->kappa[c] * mu + p->q / p->d;
                double de[3];
                factor_grid_derivs(p->pade, p->tau * lam, de);
                dg[((size_t)c * 3 + 0) * n + k] = p->tau * mu * de[0];
                dg[((size_t)c * 3 + 1) * n + k] = p->tau * p->tau * mu * de[1];
                dg[((size_t)c * 3 + 2) * n + k] = p->tau * p->tau * mu * de[2];
            }
        ETD_CUDA(cudaMemcpy(p->adj_dgrid, dg.data(), dg.size() * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<float2> dg2(dg.size());  // hi = rn(g), lo = rn(g - hi)
        for (size_t i = 0; i < dg.size(); ++i) {
            dg2[i].x = (float)dg[i];
            dg2[i].y = (float)(dg[i] - (double)dg2[i].x);
        }
        ETD_CUDA(cudaMemcpy(p->adj_dgrid2, dg2.data(), dg2.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    ETD_CUDA(cudaMemsetAsync(p->adj_acc, 0, 8 * sizeof(double), p->stream));
    s = (p->elem == 8) ? adjoint_impl<double>(p, u_ckpt, lambda_dev, n_steps)
                       : adjoint_impl<float>(p, u_ckpt, lambda_dev, n_steps);
    if (s != ETD_OK) return s;
    double acc[8];
    ETD_CUDA(cudaMemcpyAsync(acc, p->adj_acc, sizeof acc, cudaMemcpyDeviceToHost, p->stream));
    s = etd_sync(p);
    if (s != ETD_OK) return s;
    if (grad_kappa)
        for (int c = 0; c < p->ncomp; ++c) grad_kappa[c] += acc[c];
    if (grad_rx)
        for (int i = 0; i < 4; ++i) grad_rx[i] += acc[2 + i];
    return ETD_OK;
}

etd_status etd_selftest_wait_timeout(etd_plan* p, double limit_ms) {
    if (!p || p->is_batch) return fail(ETD_ERR_INVALID_ARG, "a single plan is required");
    if (!(limit_ms > 0) || limit_ms > 1000) return fail(ETD_ERR_INVALID_ARG, "limit_ms must be in (0, 1000]");
    ETD_CUDA(launch_wait_timeout_probe(p->err, limit_ms, p->stream));
    return ETD_OK;
}

etd_status etd_sync(etd_plan* p) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    for (etd_plan* g : p->groups) {
        etd_status s = etd_sync(g);
        if (s != ETD_OK) return s;
    }
    ETD_CUDA(cudaStreamSynchronize(p->stream));
    if (p->is_batch) return ETD_OK;
    unsigned flags[2] = {0, 0};
    ETD_CUDA(cudaMemcpy(flags, p->err, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[0]) {
        double saved[2] = {0, 0};
        if (flags[0] & ERR_DIVERGED) ETD_CUDA(cudaMemcpy(saved, p->stats + 4, sizeof saved, cudaMemcpyDeviceToHost));
        ETD_CUDA(cudaMemset(p->err, 0, sizeof(unsigned) * 2));
        p->uhat_valid = false;
        p->rx_ready = false;
        if (flags[0] & ERR_TIMEOUT) return fail(ETD_ERR_TIMEOUT, "a device-side wait exceeded its time limit");
        if (flags[0] & ERR_DIVERGED)
            return fail(ETD_ERR_DIVERGED,
                        "in-step field check after step %u: max |u| = %.6g (bound %.6g), %.0f non-finite values",
                        flags[1], saved[0], p->diag_max, saved[1]);
        return fail(ETD_ERR_CUDA, "device error flags 0x%x", flags[0]);
    }
    return ETD_OK;
}

// etd_step_host's result: the snapshot the next call compares against, and the
// copy out to the caller's buffer in four parts, one on the plan's stream and
// three on their own streams, so that several copy engines move it at once; the
// plan's stream waits for all four (etd_sync then covers them).
static etd_status host_copy_out(etd_plan* p, void* u_host, size_t bytes) {
    ETD_CUDA(cudaEventRecord(p->ev_out[0], p->stream));
    const size_t part = ((bytes + 3) / 4 + 4095) & ~(size_t)4095;
    for (int i = 1; i < 4; ++i) {
        const size_t off = (size_t)i * part;
        if (off >= bytes) break;
        const size_t len = bytes - off < part ? bytes - off : part;
        cudaStream_t st = p->out_stream[i - 1];
        ETD_CUDA(cudaStreamWaitEvent(st, p->ev_out[0], 0));
        ETD_CUDA(cudaMemcpyAsync(static_cast<char*>(u_host) + off, static_cast<const char*>(p->host_field) + off, len,
                                 cudaMemcpyDeviceToHost, st));
        ETD_CUDA(cudaEventRecord(p->ev_out[i], st));
    }
    ETD_CUDA(cudaMemcpyAsync(u_host, p->host_field, bytes < part ? bytes : part, cudaMemcpyDeviceToHost, p->stream));
    ETD_CUDA(cudaMemcpyAsync(p->host_snap, p->host_field, bytes, cudaMemcpyDeviceToDevice, p->stream));
    for (int i = 1; i < 4; ++i)
        if ((size_t)i * part < bytes) ETD_CUDA(cudaStreamWaitEvent(p->stream, p->ev_out[i], 0));
    return ETD_OK;
}

etd_status etd_step_host(etd_plan* p, void* u_host, int n_steps) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    if (p->is_batch) return fail(ETD_ERR_INVALID_ARG, "a batch plan is stepped with etd_batch_step");
    if (!u_host) return fail(ETD_ERR_INVALID_ARG, "u_host is NULL");
    if (n_steps < 0) return fail(ETD_ERR_INVALID_ARG, "n_steps must be >= 0");
    const size_t bytes = (size_t)p->ncomp * p->npts * p->elem;
    if (!p->host_field) {
        etd_status s = dalloc(p, &p->host_field, bytes);
        if (s == ETD_OK) s = dalloc(p, &p->host_in, bytes);
        if (s == ETD_OK) s = dalloc(p, &p->host_snap, bytes);
        if (s != ETD_OK) return s;
        ETD_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
        ETD_CUDA(cudaEventCreateWithFlags(&p->ev_host, cudaEventDisableTiming));
        for (cudaStream_t& st : p->out_stream) ETD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        for (cudaEvent_t& ev : p->ev_out) ETD_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    unsigned* const flag = reinterpret_cast<unsigned*>(p->stats + 3);
    // A caller that steps in a loop hands back the field this call returned last
    // time; then the carried spectral state still belongs to it and needs no
    // rebuild. That is taken as the likely case: the step starts at once from the
    // device copy of that field, while the incoming field is copied in and
    // compared bitwise with a snapshot of it on a second stream. If they differ
    // (the caller changed the field), the speculative step is discarded and the
    // incoming field is stepped from a rebuilt state.
    if (p->host_valid && p->uhat_valid && p->uhat_src == p->host_field && n_steps > 0) {
        ETD_CUDA(cudaEventRecord(p->ev_host, p->stream));
        ETD_CUDA(cudaStreamWaitEvent(p->copy_stream, p->ev_host, 0));
        ETD_CUDA(cudaMemcpyAsync(p->host_in, u_host, bytes, cudaMemcpyHostToDevice, p->copy_stream));
        ETD_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), p->copy_stream));
        launch_differ(p->host_in, p->host_snap, bytes, flag, p->copy_stream);
        ETD_CUDA(cudaGetLastError());
        const double t0 = p->t;
        const long long done0 = p->steps_done;
        p->host_valid = false;
        etd_status s = (p->elem == 8) ? step_impl<double>(p, p->host_field, n_steps)
                                      : step_impl<float>(p, p->host_field, n_steps);
        // read back only now: a copy into pageable host memory returns when it is
        // done, which would hold the step back if issued before it
        unsigned differ = 1;
        ETD_CUDA(cudaMemcpyAsync(&differ, flag, sizeof differ, cudaMemcpyDeviceToHost, p->copy_stream));
        ETD_CUDA(cudaStreamSynchronize(p->copy_stream));
        if (s != ETD_OK) return s;
        if (differ == 0) {
            s = host_copy_out(p, u_host, bytes);
            if (s == ETD_OK) s = etd_sync(p);
            p->host_valid = s == ETD_OK;
            return s;
        }
        // the field was changed: undo the speculative step's effects on the plan
        // (its time, step count and error flags: it stepped a field the caller no
        // longer holds)
        ETD_CUDA(cudaStreamSynchronize(p->stream));
        ETD_CUDA(cudaMemset(p->err, 0, sizeof(unsigned) * 2));
        p->t = t0;
        p->steps_done = done0;
        p->rx_ready = false;
        std::swap(p->host_in, p->host_field);
        p->uhat_valid = false;
    } else {
        ETD_CUDA(cudaMemcpyAsync(p->host_in, u_host, bytes, cudaMemcpyHostToDevice, p->stream));
        std::swap(p->host_in, p->host_field);  // step the incoming field; its state is (re)built
        p->uhat_valid = false;
    }
    p->host_valid = false;
    etd_status s = (p->elem == 8) ? step_impl<double>(p, p->host_field, n_steps)
                                  : step_impl<float>(p, p->host_field, n_steps);
    if (s != ETD_OK) return s;
    s = host_copy_out(p, u_host, bytes);
    if (s == ETD_OK) s = etd_sync(p);
    p->host_valid = s == ETD_OK;
    return s;
}

etd_status etd_transform(etd_plan* p, const void* in_dev, void* out_dev) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    if (p->is_batch) return fail(ETD_ERR_INVALID_ARG, "a batch plan is stepped with etd_batch_step");
    etd_status s = check_device_ptr(in_dev, "in_dev");
    if (s == ETD_OK) s = check_device_ptr(out_dev, "out_dev");
    if (s != ETD_OK) return s;
    int cur = 0;
    const int sp = split_for(p, p->out_slot);
    p->rx_ready = false;  // overwrites the operand buffers
    if (p->elem == 8) {
        if ((s = run_react<double>(p, -1, in_dev, p->n, p->npts, p->t, sp)) != ETD_OK) return s;
        s = run_chain<double>(p, cur, p->out_slot, EPI_PLAIN, sp, out_dev, p->n, p->npts);
    } else {
        if ((s = run_react<float>(p, -1, in_dev, p->n, p->npts, p->t, sp)) != ETD_OK) return s;
        s = run_chain<float>(p, cur, p->out_slot, EPI_PLAIN, sp, out_dev, p->n, p->npts);
    }
    return s;
}

etd_status etd_plan_invalidate(etd_plan* p) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    for (etd_plan* g : p->groups) g->uhat_valid = false;
    p->last_ptrs.clear();
    p->uhat_valid = false;
    p->uhat_src = nullptr;
    p->rx_ready = false;
    return ETD_OK;
}

etd_status etd_set_time(etd_plan* p, double t) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    if (p->is_batch) return fail(ETD_ERR_INVALID_ARG, "a batch plan is stepped with etd_batch_step");
    if (!std::isfinite(t)) return fail(ETD_ERR_INVALID_ARG, "t must be finite");
    p->t = t;
    return ETD_OK;
}

etd_status etd_field_stats(etd_plan* p, const void* u_dev, double* max_abs, long long* n_nonfinite) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    if (p->is_batch) return fail(ETD_ERR_INVALID_ARG, "a batch plan is stepped with etd_batch_step");
    if (!max_abs || !n_nonfinite) return fail(ETD_ERR_INVALID_ARG, "output pointer is NULL");
    etd_status s = check_device_ptr(u_dev, "u_dev");
    if (s != ETD_OK) return s;
    ETD_CUDA(cudaMemsetAsync(p->stats, 0, sizeof(double) * 2, p->stream));
    const long long count = (long long)p->ncomp * p->npts;
    if (p->elem == 8)
        launch_stats_f64((const double*)u_dev, count, p->stats, p->stream);
    else
        launch_stats_f32((const float*)u_dev, count, p->stats, p->stream);
    ETD_CUDA(cudaGetLastError());
    unsigned long long host[2];
    ETD_CUDA(cudaMemcpyAsync(host, p->stats, sizeof host, cudaMemcpyDeviceToHost, p->stream));
    ETD_CUDA(cudaStreamSynchronize(p->stream));
    std::memcpy(max_abs, &host[0], sizeof(double));
    *n_nonfinite = (long long)host[1];
    if (host[1]) return fail(ETD_ERR_DIVERGED, "%llu non-finite values", host[1]);
    return ETD_OK;
}

etd_status etd_get_plan_info(const etd_plan* p, etd_plan_info* info) {
    if (!p || !info) return fail(ETD_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    if (p->is_batch) {
        for (const etd_plan* g : p->groups) {
            etd_plan_info gi;
            etd_get_plan_info(g, &gi);
            info->unknowns += gi.unknowns;
            info->gemm_flops += gi.gemm_flops;
            info->step_flops += gi.step_flops;
            info->step_bytes += gi.step_bytes;
            info->products = gi.products;
            info->gemms_per_step = gi.gemms_per_step;
            info->d = gi.d;
        }
        info->n = 0;  // several grids
        info->n_comp = p->ncomp;
        info->precision = p->precision;
        info->workspace_bytes = p->workspace;
        return ETD_OK;
    }
    info->d = p->d;
    info->n = p->n;
    info->n_comp = p->ncomp;
    info->precision = p->precision;
    info->products = p->use_tc ? p->tc[0].products : (p->ozaki ? oz_pairs(p->oz_s) : 0);
    info->kernels_per_pass = (p->ozaki || p->dst) ? 2 : 1;
    info->gemms_per_step = 4 * p->d;
    info->unknowns = (long long)p->ninst * p->ncomp * p->npts;
    info->gemm_flops = 2.0 * (double)p->npts * (double)p->n * p->ncomp * p->ninst;
    info->step_flops = info->gemm_flops * info->gemms_per_step;
    info->workspace_bytes = p->workspace;
    for (int slot = 0; slot < 2; ++slot) {
        info->pass_persistent[slot] = p->use_tc && p->tc[slot].persistent ? 1 : 0;
        info->pass_tile_n[slot] = p->use_tc ? p->tc[slot].bn : 0;
    }
    // Per pass: its operand pieces and basis pieces read once; per chain of d
    // passes, d - 1 split outputs plus one final epilogue (stage 1: U^ read, Z
    // and operand pieces written; stage 2: Z read, U^+ and pieces written;
    // physical field: the field written).
    const double vals = (double)p->ninst * p->ncomp * p->npts;
    const double pin = p->use_tc ? p->tc[0].pieces : 1;
    const double opb = vals * (double)p->op_elem;
    double basis = p->dst ? 0.0 : (double)p->n * p->n * (double)p->op_elem * pin;  // DST32 reads no P
    double slicing = 0.0;
    if (p->ozaki) {
        // FP64-split: P's slices, and per pass the operand's slices written and
        // read (2 bytes each); the operand itself counts once (pin * opb), like
        // every other value, although a slicer may read a row twice (its max,
        // then its slices)
        basis = (double)p->n * p->n * 2.0 * p->oz_s;
        slicing = vals * (2.0 * 2.0 * p->oz_s);
    }
    const double st = 8.0, fe = (double)p->elem;
    const double pass_in = pin * opb + basis + slicing;
    const double split_out = pin * opb;
    const double chains = 4.0;
    info->step_bytes = chains * p->d * pass_in + chains * (p->d - 1) * split_out +
                       (vals * (st + st) + split_out) +   // stage 1: U^ read, Z written
                       (vals * (st + st) + split_out) +   // stage 2: Z read, U^+ written
                       2.0 * vals * fe;                   // two physical fields
    return ETD_OK;
}

etd_status etd_set_timing(etd_plan* p, int enable) {
    if (!p) return fail(ETD_ERR_INVALID_ARG, "plan is NULL");
    p->timing = enable != 0;
    for (etd_plan* g : p->groups) g->timing = enable != 0;
    return ETD_OK;
}

etd_status etd_kernel_times(etd_plan* p, int kind, double* total_ms, long long* launches) {
    if (!p || !total_ms || !launches) return fail(ETD_ERR_INVALID_ARG, "NULL argument");
    ETD_CUDA(cudaStreamSynchronize(p->stream));
    double ms = 0;
    long long cnt = 0;
    for (etd_plan* g : p->groups) {
        double gm = 0;
        long long gc = 0;
        etd_status s = etd_kernel_times(g, kind, &gm, &gc);
        if (s != ETD_OK) return s;
        ms += gm;
        cnt += gc;
    }
    std::vector<TimedLaunch> keep;
    for (auto& tl : p->timed) {
        if (tl.kind == kind) {
            float f = 0;
            cudaEventElapsedTime(&f, tl.a, tl.b);
            ms += f;
            ++cnt;
            p->pool.push_back(tl.a);
            p->pool.push_back(tl.b);
        } else {
            keep.push_back(tl);
        }
    }
    p->timed.swap(keep);
    *total_ms = ms;
    *launches = cnt;
    return ETD_OK;
}

etd_status etd_plan_destroy(etd_plan* p) {
    if (!p) return ETD_OK;
    for (etd_plan* g : p->groups) cudaStreamSynchronize(g->stream);
    cudaStreamSynchronize(p->stream);
    free_plan(p);
    return ETD_OK;
}

const char* etd_status_string(etd_status s) {
    switch (s) {
        case ETD_OK: return "ok";
        case ETD_ERR_INVALID_ARG: return "invalid argument";
        case ETD_ERR_OOM: return "out of device memory";
        case ETD_ERR_CUDA: return "CUDA error";
        case ETD_ERR_UNSUPPORTED: return "unsupported";
        case ETD_ERR_DIVERGED: return "non-finite values";
        case ETD_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char* etd_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
