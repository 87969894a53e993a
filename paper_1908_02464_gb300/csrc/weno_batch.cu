// Batched solver: many independent Euler problems of uneven sizes, each
// advanced to its own end time with its own CFL step, in one persistent
// launch replayed from a CUDA graph.  This file holds the 1D kernel and the
// host object shared with the 2D kernel of weno_batch2d.cu.
//
// Each CTA pulls an instance from a work queue (instances ordered largest
// first, so the tail of the schedule holds the small ones), copies it into
// three work arrays that stay L2-resident while it is being solved, and runs
// the whole RK3 loop (Sec. 4 of the paper) with block-level barriers only:
// CFL max-reduction, then per stage a chain of sweep tiles (the same
// per-tile code as the grid solver, which takes the ghost cells from the
// boundary conditions while staging, so every face is computed by identical
// arithmetic).  No CTA ever waits on another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/weno_is.h"
#include "weno_batch.cuh"
#include "weno_kernels.cuh"

namespace wis {

template <int V> struct BatchTile;
template <> struct BatchTile<0> { static constexpr int SEG = 127, NT = 128; };
template <> struct BatchTile<1> { static constexpr int SEG = 63, NT = 64; };
template <> struct BatchTile<2> { static constexpr int SEG = 255, NT = 256; };
constexpr int kBatchVariants = 3;

template <typename T, int SEG, int NT, bool EXACTDET>
__global__ void __launch_bounds__(NT) k_batch(BatchArgs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_inst;
    __shared__ double s_red[NT / 32];
    __shared__ double s_dt;
    __shared__ int s_flag;
    const T gamma = T(b.gamma);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned int k = atomicAdd(b.head, 1u);
            s_inst = k < (unsigned int)b.count ? b.order[k] : -1;
        }
        __syncthreads();
        const int inst = s_inst;
        if (inst < 0) return;
        const int n = b.n[inst];
        const long long sv = n + 6;
        T* W[3] = {reinterpret_cast<T*>(b.work0) + b.goff[inst], reinterpret_cast<T*>(b.work1) + b.goff[inst],
                   reinterpret_cast<T*>(b.work2) + b.goff[inst]};
        T* Ui = reinterpret_cast<T*>(b.U) + b.off[inst];
        for (int i = threadIdx.x; i < n; i += NT)
#pragma unroll
            for (int v = 0; v < 3; ++v) W[0][3 + v * sv + i] = Ui[(long long)v * n + i];
        const double dx = b.dx[inst], t_end = b.t_end[inst];
        // Eq. eq31
        double eps_h = b.C_thr;
        for (int k = 0; k < b.alpha_thr; ++k) eps_h *= dx / b.L_char;

        SweepArgs a;
        a.bc_lo = b.bc_lo;   // the tiles take their ghost cells from these
        a.bc_hi = b.bc_hi;
        a.acc = nullptr;
        a.mode = MODE_COMBINE;
        a.tm = nullptr;
        a.weno_count = b.weno_count;
        a.flags = nullptr;
        a.n[0] = n; a.n[1] = 1; a.n[2] = 1;
        a.sy = sv; a.sz = sv; a.sv = sv; a.off0 = 3;
        a.inv_dx = 1.0 / dx;
        a.eps_h = eps_h;
        a.gamma = b.gamma; a.eps = b.eps; a.c_lambda = b.c_lambda; a.hybrid = b.hybrid;
        a.wmode = b.wmode; a.split = b.split; a.alpha_g = nullptr;
        a.inv_dx_f = (float)(a.inv_dx * (1.0 / 60.0)); a.gamma_f = (float)b.gamma; a.eps_f = (float)b.eps;
        a.slim = sqrt(3600.0 * eps_h);
        a.slim_f = (float)a.slim; a.lam_scale_f = (float)(b.c_lambda * (1.0 / 3600.0));
        const T inv_dx_t[1] = {T(a.inv_dx)};
        const int ntiles = (n + SEG - 1) / SEG;

        int cur = 0, x = 1, y = 2;
        double t = 0.0;
        long long steps = 0;
        int status = 0;
        __syncthreads();
        const long long max_steps = b.trial_caps != nullptr ? (long long)b.trial_caps[inst] : (long long)b.max_steps;
        while (steps < max_steps) {
            // CFL max-reduction (same per-cell arithmetic as the grid solver)
            double smax = 0.0;
            bool bad = false;
            for (int i = threadIdx.x; i < n; i += NT) {
                T u[3];
#pragma unroll
                for (int v = 0; v < 3; ++v) u[v] = W[cur][3 + v * sv + i];
                T s;
                if (!cell_speed<T, 1>(u, gamma, inv_dx_t, s)) bad = true;
                else smax = maxT(smax, (double)s);
            }
            smax = warp_max(smax);
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = smax;
            const int anybad = __syncthreads_or(bad);
            if (threadIdx.x == 0) {
                double m = 0.0;
                for (int w = 0; w < NT / 32; ++w) m = maxT(m, s_red[w]);
                int clipped = 0;
                s_dt = anybad ? 0.0 : cfl_step(b.cfl, m, t, t_end, &clipped);
                s_flag = clipped;
            }
            __syncthreads();
            const double dt = s_dt;
            const int clipped = s_flag;
            if (anybad) { status = WENO_ERR_NONPHYSICAL; break; }
            if (!(dt > 0.0)) break;
            const T dtt = T(dt);
            // three stages: x = cur + dt L(cur); y = 3/4 cur + 1/4 (x + dt L(x));
            // x = 1/3 cur + 2/3 (y + dt L(y))
            const int in_[3] = {cur, x, y}, out_[3] = {x, y, x};
            const double ra[3] = {0.0, 0.75, 1.0 / 3.0}, rb[3] = {1.0, 0.25, 2.0 / 3.0};
            bool sbad = false;
            for (int st = 0; st < 3; ++st) {
                a.U = W[in_[st]];
                a.Un = W[cur];
                a.out = W[out_[st]];
                a.rk_a = ra[st]; a.rk_b = rb[st];
                a.rk_a_f = (float)ra[st]; a.rk_b_f = (float)rb[st];
                for (int tile = 0; tile < ntiles; ++tile)
                    sbad |= sweep_tile<T, 1, 0, 1, SEG, NT, EXACTDET>(a, tile, 0, 0, dtt, smem_raw);
            }
            if (__syncthreads_or(sbad)) { status = WENO_ERR_NONPHYSICAL; break; }
            const int tmp = cur;
            cur = x;
            x = tmp;
            t = clipped ? t_end : t + dt;
            ++steps;
        }
        if (b.write_back)
            for (int i = threadIdx.x; i < n; i += NT)
#pragma unroll
                for (int v = 0; v < 3; ++v) Ui[(long long)v * n + i] = W[cur][3 + v * sv + i];
        if (threadIdx.x == 0) {
            b.status[inst] = status;
            b.steps[inst] = steps;
            b.t_out[inst] = t;
        }
        __syncthreads();
    }
}

template <typename T, bool EXACTDET, int V>
cudaError_t batch_config(int* blocks_per_sm, size_t* smem)
{
    using BT = BatchTile<V>;
    using SM = SweepSmem<T, 1, 1, BT::SEG>;
    auto kern = k_batch<T, BT::SEG, BT::NT, EXACTDET>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    *smem = SM::bytes;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, BT::NT, SM::bytes);
}

template <typename T, bool EXACTDET, int V>
cudaError_t batch_launch(const BatchArgs& b, int blocks, cudaStream_t s)
{
    using BT = BatchTile<V>;
    using SM = SweepSmem<T, 1, 1, BT::SEG>;
    k_batch<T, BT::SEG, BT::NT, EXACTDET><<<blocks, BT::NT, SM::bytes, s>>>(b);
    return cudaGetLastError();
}

}  // namespace wis

using wis::BatchArgs;

struct weno_batch {
    int dim = 1;   // 1: [3][n] instances (k_batch); 2: [4][ny][nx] instances (k_batch2d)
    int count = 0, prec = 0, dev = 0, nsm = 1;
    size_t esz = 8;
    weno_params p;
    int bc_lo = 0, bc_hi = 0, max_steps = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    long long total_cells = 0, total_ghosted = 0;
    int* order = nullptr;
    int* n = nullptr;
    long long* off = nullptr;
    long long* goff = nullptr;
    double* dx = nullptr;
    double* t_end = nullptr;
    int* ny = nullptr;        // 2D
    double* dy = nullptr;     // 2D
    int bc_lo_y = 0, bc_hi_y = 0;
    void* work[4] = {nullptr, nullptr, nullptr, nullptr};   // the fourth: 2D accumulator
    int* status = nullptr;
    long long* steps = nullptr;
    double* t_out = nullptr;
    unsigned int* head = nullptr;
    unsigned long long* wcount = nullptr;
    int* trial_caps = nullptr;
    std::vector<int> n_host;      // steps grow with this size: n (1D), max(nx, ny) (2D)
    int variant = 0;
    int blocks = 0;
    cudaGraphExec_t graph = nullptr;
    void* graph_U = nullptr;
    std::string err;
};

static std::string g_batch_err;

#define BCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            bt->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return WENO_ERR_CUDA;                                                           \
        }                                                                                   \
    } while (0)

static cudaError_t batch_dispatch_config(int dim, int prec, int v, int* bps, size_t* smem)
{
    using namespace wis;
    if (dim == 2) return batch2d_config(prec, v, bps, smem);
    if (prec == WENO_FP64) {
        if (v == 1) return batch_config<double, false, 1>(bps, smem);
        if (v == 2) return batch_config<double, false, 2>(bps, smem);
        return batch_config<double, false, 0>(bps, smem);
    }
    const bool ex = prec == WENO_MIXED;
    if (v == 1) return ex ? batch_config<float, true, 1>(bps, smem) : batch_config<float, false, 1>(bps, smem);
    if (v == 2) return ex ? batch_config<float, true, 2>(bps, smem) : batch_config<float, false, 2>(bps, smem);
    return ex ? batch_config<float, true, 0>(bps, smem) : batch_config<float, false, 0>(bps, smem);
}

static cudaError_t batch_dispatch_launch(int dim, int prec, int v, const BatchArgs& b, int blocks, cudaStream_t s)
{
    using namespace wis;
    if (dim == 2) return batch2d_launch(prec, v, b, blocks, s);
    if (prec == WENO_FP64) {
        if (v == 1) return batch_launch<double, false, 1>(b, blocks, s);
        if (v == 2) return batch_launch<double, false, 2>(b, blocks, s);
        return batch_launch<double, false, 0>(b, blocks, s);
    }
    const bool ex = prec == WENO_MIXED;
    if (v == 1) return ex ? batch_launch<float, true, 1>(b, blocks, s) : batch_launch<float, false, 1>(b, blocks, s);
    if (v == 2) return ex ? batch_launch<float, true, 2>(b, blocks, s) : batch_launch<float, false, 2>(b, blocks, s);
    return ex ? batch_launch<float, true, 0>(b, blocks, s) : batch_launch<float, false, 0>(b, blocks, s);
}

static BatchArgs batch_args(weno_batch* bt, void* U, int max_steps, int write_back)
{
    BatchArgs b;
    std::memset(&b, 0, sizeof(b));
    b.count = bt->count;
    b.order = bt->order; b.n = bt->n; b.off = bt->off; b.goff = bt->goff;
    b.dx = bt->dx; b.t_end = bt->t_end;
    b.U = U;
    b.work0 = bt->work[0]; b.work1 = bt->work[1]; b.work2 = bt->work[2];
    b.status = bt->status; b.steps = bt->steps; b.t_out = bt->t_out;
    b.head = bt->head;
    b.weno_count = bt->wcount;
    b.max_steps = max_steps;
    b.write_back = write_back;
    b.gamma = bt->p.gamma; b.cfl = bt->p.cfl; b.eps = bt->p.eps; b.c_lambda = bt->p.c_lambda;
    b.C_thr = bt->p.C_thr; b.L_char = bt->p.L_char; b.alpha_thr = bt->p.alpha_thr; b.hybrid = bt->p.hybrid;
    b.bc_lo = bt->bc_lo; b.bc_hi = bt->bc_hi;
    b.wmode = bt->p.weights; b.split = bt->p.splitting;
    b.ny = bt->ny; b.dy = bt->dy;
    b.bc_lo_y = bt->bc_lo_y; b.bc_hi_y = bt->bc_hi_y;
    b.work3 = bt->work[3];
    return b;
}

static weno_status set_variant(weno_batch* bt, int v, int blocks_per_sm_cap)
{
    int bps = 0;
    size_t smem = 0;
    BCK(batch_dispatch_config(bt->dim, bt->prec, v, &bps, &smem));
    if (bps < 1) { bt->err = "batch kernel cannot be resident"; return WENO_ERR_CUDA; }
    if (blocks_per_sm_cap > 0 && bps > blocks_per_sm_cap) bps = blocks_per_sm_cap;
    bt->variant = v;
    long long blocks = (long long)bps * bt->nsm;
    if (blocks > bt->count) blocks = bt->count;
    bt->blocks = (int)blocks;
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    bt->graph = nullptr;
    return WENO_OK;
}

// reset the queue and launch once (on stream s, optionally under capture)
static cudaError_t enqueue_run(weno_batch* bt, void* U, int max_steps, int write_back, cudaStream_t s,
                               const int* trial_caps = nullptr)
{
    cudaError_t e = cudaMemsetAsync(bt->head, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    BatchArgs b = batch_args(bt, U, max_steps, write_back);
    b.trial_caps = trial_caps;
    return batch_dispatch_launch(bt->dim, bt->prec, bt->variant, b, bt->blocks, s);
}

static void batch_free(weno_batch* bt)
{
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    void* ptrs[] = {bt->order, bt->n, bt->off, bt->goff, bt->dx, bt->t_end, bt->work[0], bt->work[1],
                    bt->work[2], bt->work[3], bt->status, bt->steps, bt->t_out, bt->head, bt->wcount,
                    bt->trial_caps, bt->ny, bt->dy};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (bt->cap) cudaStreamDestroy(bt->cap);
}

extern "C" {

weno_status weno_batch_create(const weno_batch_desc* d, const weno_params* params, void* stream, weno_batch** out)
{
    if (out) *out = nullptr;
    if (!d || !params || !out || d->count < 1 || !d->n || !d->lo || !d->hi || !d->t_end) {
        g_batch_err = "invalid batch description";
        return WENO_ERR_INVALID_ARG;
    }
    if (params->precision < WENO_FP64 || params->precision > WENO_MIXED || d->max_steps < 0 ||
        params->weights < 0 || params->weights > 3 || params->splitting < 0 || params->splitting > 2) {
        g_batch_err = "invalid precision, weights, splitting or max_steps";
        return WENO_ERR_INVALID_ARG;
    }
    if (params->splitting == 1) {
        g_batch_err = "global Lax-Friedrichs splitting is not available for batches (use LLF or Roe)";
        return WENO_ERR_UNSUPPORTED;
    }
    for (int s = 0; s < 2; ++s) {
        const int bc = s == 0 ? d->bc_lo : d->bc_hi;
        if (bc != WENO_BC_TRANSMISSIVE && bc != WENO_BC_REFLECT && bc != WENO_BC_PERIODIC) {
            g_batch_err = "batched problems take transmissive, reflecting or periodic boundaries";
            return WENO_ERR_INVALID_ARG;
        }
    }
    if ((d->bc_lo == WENO_BC_PERIODIC) != (d->bc_hi == WENO_BC_PERIODIC)) {
        g_batch_err = "periodic boundaries must be paired";
        return WENO_ERR_INVALID_ARG;
    }
    const int cnt = d->count;
    std::vector<long long> off(cnt), goff(cnt);
    std::vector<double> dx(cnt), tend(cnt);
    long long tc = 0, tg = 0;
    for (int i = 0; i < cnt; ++i) {
        if (d->n[i] < 3 || !(d->hi[i] > d->lo[i]) || !(d->t_end[i] >= 0.0)) {
            g_batch_err = "instance with n < 3, hi <= lo or negative t_end";
            return WENO_ERR_INVALID_ARG;
        }
        off[i] = tc;
        goff[i] = tg;
        tc += 3LL * d->n[i];
        tg += 3LL * (d->n[i] + 6);
        dx[i] = (d->hi[i] - d->lo[i]) / d->n[i];
        tend[i] = d->t_end[i];
    }
    // schedule: largest instances first
    std::vector<int> order(cnt);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d->n[a] > d->n[b]; });

    weno_batch* bt = new (std::nothrow) weno_batch();
    if (!bt) { g_batch_err = "out of host memory"; return WENO_ERR_CUDA; }
    bt->count = cnt;
    bt->p = *params;
    bt->prec = params->precision;
    bt->esz = bt->prec == WENO_FP64 ? sizeof(double) : sizeof(float);
    bt->bc_lo = d->bc_lo;
    bt->bc_hi = d->bc_hi;
    bt->max_steps = d->max_steps > 0 ? d->max_steps : 0x7fffffff;
    bt->stream = (cudaStream_t)stream;
    bt->total_cells = tc / 3;
    bt->total_ghosted = tg;
    cudaError_t e = cudaGetDevice(&bt->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bt->nsm, cudaDevAttrMultiProcessorCount, bt->dev);
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void**)&bt->order, sizeof(int) * cnt);
    alloc((void**)&bt->n, sizeof(int) * cnt);
    alloc((void**)&bt->off, sizeof(long long) * cnt);
    alloc((void**)&bt->goff, sizeof(long long) * cnt);
    alloc((void**)&bt->dx, sizeof(double) * cnt);
    alloc((void**)&bt->t_end, sizeof(double) * cnt);
    for (int k = 0; k < 3; ++k) alloc(&bt->work[k], bt->esz * (size_t)tg);
    alloc((void**)&bt->status, sizeof(int) * cnt);
    alloc((void**)&bt->steps, sizeof(long long) * cnt);
    alloc((void**)&bt->t_out, sizeof(double) * cnt);
    alloc((void**)&bt->head, sizeof(unsigned int));
    alloc((void**)&bt->wcount, sizeof(unsigned long long));
    alloc((void**)&bt->trial_caps, sizeof(int) * cnt);
    bt->n_host.assign(d->n, d->n + cnt);
    if (e == cudaSuccess) e = cudaMemcpy(bt->order, order.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->n, d->n, sizeof(int) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->off, off.data(), sizeof(long long) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->goff, goff.data(), sizeof(long long) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->dx, dx.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->t_end, tend.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(bt->wcount, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        g_batch_err = std::string("weno_batch_create: ") + cudaGetErrorString(e);
        batch_free(bt);
        delete bt;
        return WENO_ERR_CUDA;
    }
    weno_status st = set_variant(bt, 0, 0);
    if (st != WENO_OK) {
        g_batch_err = bt->err;
        batch_free(bt);
        delete bt;
        return st;
    }
    *out = bt;
    return WENO_OK;
}

weno_status weno_batch2d_create(const weno_batch2d_desc* d, const weno_params* params, void* stream,
                                weno_batch** out)
{
    if (out) *out = nullptr;
    if (!d || !params || !out || d->count < 1 || !d->nx || !d->ny || !d->lo_x || !d->hi_x || !d->lo_y ||
        !d->hi_y || !d->t_end) {
        g_batch_err = "invalid 2D batch description";
        return WENO_ERR_INVALID_ARG;
    }
    if (params->precision < WENO_FP64 || params->precision > WENO_MIXED || d->max_steps < 0 ||
        params->weights < 0 || params->weights > 3 || params->splitting < 0 || params->splitting > 2) {
        g_batch_err = "invalid precision, weights, splitting or max_steps";
        return WENO_ERR_INVALID_ARG;
    }
    if (params->splitting == 1) {
        g_batch_err = "global Lax-Friedrichs splitting is not available for batches (use LLF or Roe)";
        return WENO_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < 2; ++a) {
        for (int s = 0; s < 2; ++s) {
            const int bc = s == 0 ? d->bc_lo[a] : d->bc_hi[a];
            if (bc != WENO_BC_TRANSMISSIVE && bc != WENO_BC_REFLECT && bc != WENO_BC_PERIODIC) {
                g_batch_err = "batched problems take transmissive, reflecting or periodic boundaries";
                return WENO_ERR_INVALID_ARG;
            }
        }
        if ((d->bc_lo[a] == WENO_BC_PERIODIC) != (d->bc_hi[a] == WENO_BC_PERIODIC)) {
            g_batch_err = "periodic boundaries must be paired";
            return WENO_ERR_INVALID_ARG;
        }
    }
    const int cnt = d->count;
    std::vector<long long> off(cnt);
    std::vector<double> dx(cnt), dy(cnt), tend(cnt), work(cnt);
    std::vector<int> lin(cnt);
    long long tc = 0;
    for (int i = 0; i < cnt; ++i) {
        if (d->nx[i] < 3 || d->ny[i] < 3 || !(d->hi_x[i] > d->lo_x[i]) || !(d->hi_y[i] > d->lo_y[i]) ||
            !(d->t_end[i] >= 0.0)) {
            g_batch_err = "instance with nx or ny < 3, hi <= lo or negative t_end";
            return WENO_ERR_INVALID_ARG;
        }
        off[i] = tc;
        tc += 4LL * d->nx[i] * d->ny[i];
        dx[i] = (d->hi_x[i] - d->lo_x[i]) / d->nx[i];
        dy[i] = (d->hi_y[i] - d->lo_y[i]) / d->ny[i];
        tend[i] = d->t_end[i];
        lin[i] = std::max(d->nx[i], d->ny[i]);
        // work of a run ~ cells x steps, and the steps grow with the finer spacing
        work[i] = (double)d->nx[i] * d->ny[i] * lin[i];
    }
    // schedule: most work first
    std::vector<int> order(cnt);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });

    weno_batch* bt = new (std::nothrow) weno_batch();
    if (!bt) { g_batch_err = "out of host memory"; return WENO_ERR_CUDA; }
    bt->dim = 2;
    bt->count = cnt;
    bt->p = *params;
    bt->prec = params->precision;
    bt->esz = bt->prec == WENO_FP64 ? sizeof(double) : sizeof(float);
    bt->bc_lo = d->bc_lo[0];
    bt->bc_hi = d->bc_hi[0];
    bt->bc_lo_y = d->bc_lo[1];
    bt->bc_hi_y = d->bc_hi[1];
    bt->max_steps = d->max_steps > 0 ? d->max_steps : 0x7fffffff;
    bt->stream = (cudaStream_t)stream;
    bt->total_cells = tc / 4;
    bt->total_ghosted = tc;
    cudaError_t e = cudaGetDevice(&bt->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bt->nsm, cudaDevAttrMultiProcessorCount, bt->dev);
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void**)&bt->order, sizeof(int) * cnt);
    alloc((void**)&bt->n, sizeof(int) * cnt);
    alloc((void**)&bt->ny, sizeof(int) * cnt);
    alloc((void**)&bt->off, sizeof(long long) * cnt);
    alloc((void**)&bt->goff, sizeof(long long) * cnt);
    alloc((void**)&bt->dx, sizeof(double) * cnt);
    alloc((void**)&bt->dy, sizeof(double) * cnt);
    alloc((void**)&bt->t_end, sizeof(double) * cnt);
    for (int k = 0; k < 4; ++k) alloc(&bt->work[k], bt->esz * (size_t)tc);
    alloc((void**)&bt->status, sizeof(int) * cnt);
    alloc((void**)&bt->steps, sizeof(long long) * cnt);
    alloc((void**)&bt->t_out, sizeof(double) * cnt);
    alloc((void**)&bt->head, sizeof(unsigned int));
    alloc((void**)&bt->wcount, sizeof(unsigned long long));
    alloc((void**)&bt->trial_caps, sizeof(int) * cnt);
    bt->n_host = lin;
    if (e == cudaSuccess) e = cudaMemcpy(bt->order, order.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->n, d->nx, sizeof(int) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->ny, d->ny, sizeof(int) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->off, off.data(), sizeof(long long) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->goff, off.data(), sizeof(long long) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->dx, dx.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->dy, dy.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->t_end, tend.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(bt->wcount, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        g_batch_err = std::string("weno_batch2d_create: ") + cudaGetErrorString(e);
        batch_free(bt);
        delete bt;
        return WENO_ERR_CUDA;
    }
    weno_status st = set_variant(bt, 0, 0);
    if (st != WENO_OK) {
        g_batch_err = bt->err;
        batch_free(bt);
        delete bt;
        return st;
    }
    *out = bt;
    return WENO_OK;
}

void weno_batch_destroy(weno_batch* bt)
{
    if (!bt) return;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    else cudaDeviceSynchronize();
    batch_free(bt);
    delete bt;
}

const char* weno_batch_last_error(const weno_batch* bt) { return bt ? bt->err.c_str() : g_batch_err.c_str(); }

weno_status weno_batch_run(weno_batch* bt, void* U_dev)
{
    if (!bt || !U_dev) return WENO_ERR_INVALID_ARG;
    if (!bt->graph || bt->graph_U != U_dev) {
        if (bt->graph) cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeRelaxed));
        cudaError_t e = enqueue_run(bt, U_dev, bt->max_steps, 1, bt->cap);
        cudaError_t e2 = cudaStreamEndCapture(bt->cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            bt->err = std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
            return WENO_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&bt->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            bt->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
            return WENO_ERR_CUDA;
        }
        bt->graph_U = U_dev;
    }
    BCK(cudaGraphLaunch(bt->graph, bt->stream));
    return WENO_OK;
}

weno_status weno_batch_results(weno_batch* bt, int* status, long long* steps, double* t)
{
    if (!bt) return WENO_ERR_INVALID_ARG;
    if (status) BCK(cudaMemcpyAsync(status, bt->status, sizeof(int) * bt->count, cudaMemcpyDeviceToHost, bt->stream));
    if (steps) BCK(cudaMemcpyAsync(steps, bt->steps, sizeof(long long) * bt->count, cudaMemcpyDeviceToHost, bt->stream));
    if (t) BCK(cudaMemcpyAsync(t, bt->t_out, sizeof(double) * bt->count, cudaMemcpyDeviceToHost, bt->stream));
    BCK(cudaStreamSynchronize(bt->stream));
    if (status)
        for (int i = 0; i < bt->count; ++i)
            if (status[i] != WENO_OK) {
                bt->err = "at least one instance reached a non-physical state";
                return WENO_ERR_NONPHYSICAL;
            }
    return WENO_OK;
}

weno_status weno_batch_weno_face_count(weno_batch* bt, unsigned long long* count, int reset)
{
    if (!bt) return WENO_ERR_INVALID_ARG;
    unsigned long long v = 0;
    BCK(cudaMemcpyAsync(&v, bt->wcount, sizeof(v), cudaMemcpyDeviceToHost, bt->stream));
    BCK(cudaStreamSynchronize(bt->stream));
    if (count) *count = v;
    if (reset) {
        BCK(cudaMemsetAsync(bt->wcount, 0, sizeof(unsigned long long), bt->stream));
        BCK(cudaStreamSynchronize(bt->stream));
    }
    return WENO_OK;
}

weno_status weno_batch_set_config(weno_batch* bt, int variant, int blocks_per_sm, int* blocks)
{
    if (!bt) return WENO_ERR_INVALID_ARG;
    if (variant < 0 || variant >= (bt->dim == 2 ? wis::kBatch2Variants : wis::kBatchVariants) || blocks_per_sm < 0) {
        bt->err = "set_config: variant must be 0, 1 or 2 and blocks_per_sm >= 0";
        return WENO_ERR_INVALID_ARG;
    }
    const weno_status st = set_variant(bt, variant, blocks_per_sm);
    if (st == WENO_OK && blocks) *blocks = bt->blocks;
    return st;
}

weno_status weno_batch_autotune(weno_batch* bt, const void* U_dev, int trial_steps, int* choice)
{
    if (!bt || !U_dev || trial_steps < 1) return WENO_ERR_INVALID_ARG;
    // trial steps per instance in proportion to its cells: a full run's step
    // count grows with the cell count (the CFL step shrinks with dx), so its
    // work grows like N^2, and the trial keeps that shape
    const int nmax = *std::max_element(bt->n_host.begin(), bt->n_host.end());
    std::vector<int> tc(bt->count);
    for (int i = 0; i < bt->count; ++i)
        tc[i] = std::max(1, (int)std::ceil((double)trial_steps * bt->n_host[i] / nmax));
    BCK(cudaMemcpy(bt->trial_caps, tc.data(), sizeof(int) * bt->count, cudaMemcpyHostToDevice));
    // the trials start from a scratch copy advanced to half of each
    // instance's end time: the cost of a step depends on how far the waves
    // have spread, and trials from the initial jumps rank the configurations
    // unlike full runs do (they favour small tiles that lose on developed
    // solutions)
    const size_t sbytes = (size_t)bt->total_cells * (bt->dim + 2) * bt->esz;
    void* Us = nullptr;
    double* t_half = nullptr;
    BCK(cudaMalloc(&Us, sbytes));
    if (cudaMalloc(&t_half, sizeof(double) * bt->count) != cudaSuccess) {
        cudaFree(Us);
        bt->err = "autotune: out of device memory";
        return WENO_ERR_CUDA;
    }
    std::vector<double> th(bt->count);
    cudaError_t ce = cudaMemcpy(th.data(), bt->t_end, sizeof(double) * bt->count, cudaMemcpyDeviceToHost);
    for (double& x : th) x *= 0.5;
    if (ce == cudaSuccess)
        ce = cudaMemcpy(t_half, th.data(), sizeof(double) * bt->count, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(Us, U_dev, sbytes, cudaMemcpyDeviceToDevice, bt->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(bt->head, 0, sizeof(unsigned int), bt->stream);
    if (ce == cudaSuccess) {
        BatchArgs b = batch_args(bt, Us, bt->max_steps, 1);
        b.t_end = t_half;
        ce = batch_dispatch_launch(bt->dim, bt->prec, bt->variant, b, bt->blocks, bt->stream);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(bt->stream);
    cudaFree(t_half);
    if (ce != cudaSuccess) {
        cudaFree(Us);
        bt->err = std::string("autotune: developing the trial state: ") + cudaGetErrorString(ce);
        return WENO_ERR_CUDA;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) { cudaFree(Us); bt->err = "cudaEventCreate"; return WENO_ERR_CUDA; }
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0); cudaFree(Us); bt->err = "cudaEventCreate"; return WENO_ERR_CUDA;
    }
    float best = 1e30f;
    int best_v = bt->variant, best_cap = 0;
    const int caps[3] = {0, 4, 2};   // 0 = as many CTAs per SM as fit
    weno_status st = WENO_OK;
    const int nvariants = bt->dim == 2 ? wis::kBatch2Variants : wis::kBatchVariants;
    for (int v = 0; v < nvariants && st == WENO_OK; ++v) {
        for (int c = 0; c < 3 && st == WENO_OK; ++c) {
            st = set_variant(bt, v, caps[c]);
            if (st != WENO_OK) break;
            float ms = 1e30f;
            for (int r = 0; r < 2; ++r) {   // first run loads the kernel
                if (cudaEventRecord(e0, bt->stream) != cudaSuccess ||
                    enqueue_run(bt, Us, trial_steps, 0, bt->stream, bt->trial_caps) != cudaSuccess ||
                    cudaEventRecord(e1, bt->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    bt->err = "batch autotune launch failed";
                    st = WENO_ERR_CUDA;
                    break;
                }
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (st == WENO_OK && ms < best) { best = ms; best_v = v; best_cap = caps[c]; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(Us);
    if (st != WENO_OK) return st;
    st = set_variant(bt, best_v, best_cap);
    if (choice) { choice[0] = best_v; choice[1] = bt->blocks; }
    return st;
}

weno_status weno_batch_solve(const weno_batch_desc* d, const weno_params* params, void* stream, void* U_dev,
                             int* per_instance)
{
    weno_batch* bt = nullptr;
    weno_status st = weno_batch_create(d, params, stream, &bt);
    if (st != WENO_OK) return st;
    st = weno_batch_run(bt, U_dev);
    if (st == WENO_OK) st = weno_batch_results(bt, per_instance, nullptr, nullptr);
    if (st != WENO_OK && st != WENO_ERR_NONPHYSICAL) g_batch_err = bt->err;
    weno_batch_destroy(bt);
    return st;
}

}  // extern "C"
