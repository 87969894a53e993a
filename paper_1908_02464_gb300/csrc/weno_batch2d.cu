// Batched 2D solver: many independent 2D Euler problems of uneven sizes, each
// advanced to its own end time with its own CFL step, in one persistent
// launch (replayed from a CUDA graph by the host code in weno_batch.cu).
//
// A CTA takes an instance from the work queue (largest first), copies its
// state into work arrays that stay L2-resident while it is being solved, and
// runs the whole RK3 loop (Sec. 4 of the paper) alone, with block-level
// barriers only.  Each stage is the grid solver's pair of sweeps: the y
// sweep writes its flux divergence (Eq. goveq5) to an accumulator, then the
// x sweep adds its own and applies the RK3 combination.  Both sweeps are
// chains of the grid solver's tiles (sweep_tile), whose ghost cells come
// from the boundary conditions while staging, so every face is computed by
// the same arithmetic as in the single-problem solver.
#include <cuda_runtime.h>

#include "../../include/weno_is.h"
#include "weno_batch.cuh"
#include "weno_kernels.cuh"

namespace wis {

// Tile shapes (LINES x SEG, LINES (SEG + 1) faces = CTA size) of the x and y
// sweeps.  Batched instances have short lines (tens of cells), so the tiles
// hold several lines; the y tiles hold 8 or 4 x-adjacent columns, so that
// their loads are row pieces.
template <int V> struct Batch2Tile;
template <> struct Batch2Tile<0> { static constexpr int NT = 128, XL = 4, XS = 31, YL = 8, YS = 15; };
template <> struct Batch2Tile<1> { static constexpr int NT = 128, XL = 2, XS = 63, YL = 4, YS = 31; };
template <> struct Batch2Tile<2> { static constexpr int NT = 64, XL = 2, XS = 31, YL = 4, YS = 15; };

template <typename T, int V>
struct Batch2Smem {
    using BT = Batch2Tile<V>;
    static constexpr size_t X = SweepSmem<T, 2, BT::XL, BT::XS>::bytes;
    static constexpr size_t Y = SweepSmem<T, 2, BT::YL, BT::YS>::bytes;
    static constexpr size_t bytes = X > Y ? X : Y;
};

// sweep arguments of direction d (0 = x, 1 = y) of one instance; the work
// arrays hold the interior only, [4][ny][nx] (ghost cells are computed while
// staging the tiles)
__device__ __forceinline__ void batch2d_dir_args(const BatchArgs& b, int d, int nx, int ny, double h, SweepArgs& a)
{
    a.n[0] = nx; a.n[1] = ny; a.n[2] = 1;
    a.sy = nx; a.sz = (long long)nx * ny; a.sv = (long long)nx * ny; a.off0 = 0;
    a.acc = nullptr; a.Un = nullptr; a.out = nullptr;
    a.tm = nullptr;
    a.weno_count = b.weno_count;
    a.flags = nullptr;
    a.alpha_g = nullptr;
    a.inv_dx = 1.0 / h;
    // Eq. eq31: eps_h = C (h / L)^alpha with the spacing of the sweep direction
    double eps_h = b.C_thr;
    for (int k = 0; k < b.alpha_thr; ++k) eps_h *= h / b.L_char;
    a.eps_h = eps_h;
    a.gamma = b.gamma; a.eps = b.eps; a.c_lambda = b.c_lambda; a.hybrid = b.hybrid;
    a.wmode = b.wmode; a.split = b.split;
    a.inv_dx_f = (float)(a.inv_dx * (1.0 / 60.0));
    a.gamma_f = (float)b.gamma; a.eps_f = (float)b.eps;
    a.slim = sqrt(3600.0 * eps_h);
    a.slim_f = (float)a.slim;
    a.lam_scale_f = (float)(b.c_lambda * (1.0 / 3600.0));
    a.bc_lo = d == 0 ? b.bc_lo : b.bc_lo_y;
    a.bc_hi = d == 0 ? b.bc_hi : b.bc_hi_y;
    a.stage = 0;
    a.xs_fixed = 0.0;
}

template <typename T, int V, bool EXACTDET>
__global__ void __launch_bounds__(Batch2Tile<V>::NT) k_batch2d(BatchArgs b)
{
    using BT = Batch2Tile<V>;
    constexpr int NT = BT::NT;
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
        const int nx = b.n[inst], ny = b.ny[inst];
        const long long cells = (long long)nx * ny;
        T* W[3] = {reinterpret_cast<T*>(b.work0) + b.goff[inst], reinterpret_cast<T*>(b.work1) + b.goff[inst],
                   reinterpret_cast<T*>(b.work2) + b.goff[inst]};
        T* acc = reinterpret_cast<T*>(b.work3) + b.goff[inst];
        T* Ui = reinterpret_cast<T*>(b.U) + b.off[inst];
        for (long long i = threadIdx.x; i < 4 * cells; i += NT) W[0][i] = Ui[i];
        const double dx = b.dx[inst], dy = b.dy[inst], t_end = b.t_end[inst];
        SweepArgs ax, ay;
        batch2d_dir_args(b, 0, nx, ny, dx, ax);
        batch2d_dir_args(b, 1, nx, ny, dy, ay);
        ay.mode = MODE_ACC_SET;
        ay.acc = acc;
        ax.mode = MODE_COMBINE;
        ax.acc = acc;
        ax.acc_scale = ay.inv_dx * (1.0 / 60.0);   // the y-sweep stores unscaled flux differences
        ax.acc_scale_f = (float)ax.acc_scale;
        const T inv_dx_t[2] = {T(ax.inv_dx), T(ay.inv_dx)};
        const int nsx = (nx + BT::XS - 1) / BT::XS, nlx = (ny + BT::XL - 1) / BT::XL;
        const int nsy = (ny + BT::YS - 1) / BT::YS, nly = (nx + BT::YL - 1) / BT::YL;

        int cur = 0, x = 1, y = 2;
        double t = 0.0;
        long long steps = 0;
        int status = 0;
        __syncthreads();
        const long long max_steps = b.trial_caps != nullptr ? (long long)b.trial_caps[inst] : (long long)b.max_steps;
        while (steps < max_steps) {
            // CFL max-reduction (the grid solver's per-cell arithmetic)
            double smax = 0.0;
            bool bad = false;
            for (long long i = threadIdx.x; i < cells; i += NT) {
                T u[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) u[v] = W[cur][v * cells + i];
                T s;
                if (!cell_speed<T, 2>(u, gamma, inv_dx_t, s)) bad = true;
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
                ay.U = W[in_[st]];
                for (int tile = 0; tile < nsy * nly; ++tile) {
                    const int seg = tile % nsy, lg = tile / nsy;
                    sweep_tile<T, 2, 1, BT::YL, BT::YS, NT, EXACTDET>(ay, seg, lg * BT::YL, 0, dtt, smem_raw);
                }
                ax.U = W[in_[st]];
                ax.Un = W[cur];
                ax.out = W[out_[st]];
                ax.rk_a = ra[st]; ax.rk_b = rb[st];
                ax.rk_a_f = (float)ra[st]; ax.rk_b_f = (float)rb[st];
                for (int tile = 0; tile < nsx * nlx; ++tile) {
                    const int seg = tile % nsx, lg = tile / nsx;
                    sbad |= sweep_tile<T, 2, 0, BT::XL, BT::XS, NT, EXACTDET>(ax, seg, lg * BT::XL, 0, dtt,
                                                                              smem_raw);
                }
            }
            if (__syncthreads_or(sbad)) { status = WENO_ERR_NONPHYSICAL; break; }
            const int tmp = cur;
            cur = x;
            x = tmp;
            t = clipped ? t_end : t + dt;
            ++steps;
        }
        if (b.write_back)
            for (long long i = threadIdx.x; i < 4 * cells; i += NT) Ui[i] = W[cur][i];
        if (threadIdx.x == 0) {
            b.status[inst] = status;
            b.steps[inst] = steps;
            b.t_out[inst] = t;
        }
        __syncthreads();
    }
}

template <typename T, bool EXACTDET, int V>
static cudaError_t config_v(int* blocks_per_sm, size_t* smem)
{
    using SM = Batch2Smem<T, V>;
    auto kern = k_batch2d<T, V, EXACTDET>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    *smem = SM::bytes;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, Batch2Tile<V>::NT, SM::bytes);
}

template <typename T, bool EXACTDET, int V>
static cudaError_t launch_v(const BatchArgs& b, int blocks, cudaStream_t s)
{
    k_batch2d<T, V, EXACTDET><<<blocks, Batch2Tile<V>::NT, Batch2Smem<T, V>::bytes, s>>>(b);
    return cudaGetLastError();
}

template <typename T, bool EXACTDET>
static cudaError_t config_t(int v, int* bps, size_t* smem)
{
    if (v == 1) return config_v<T, EXACTDET, 1>(bps, smem);
    if (v == 2) return config_v<T, EXACTDET, 2>(bps, smem);
    return config_v<T, EXACTDET, 0>(bps, smem);
}

template <typename T, bool EXACTDET>
static cudaError_t launch_t(int v, const BatchArgs& b, int blocks, cudaStream_t s)
{
    if (v == 1) return launch_v<T, EXACTDET, 1>(b, blocks, s);
    if (v == 2) return launch_v<T, EXACTDET, 2>(b, blocks, s);
    return launch_v<T, EXACTDET, 0>(b, blocks, s);
}

cudaError_t batch2d_config(int prec, int v, int* blocks_per_sm, size_t* smem)
{
    if (prec == WENO_FP64) return config_t<double, false>(v, blocks_per_sm, smem);
    if (prec == WENO_MIXED) return config_t<float, true>(v, blocks_per_sm, smem);
    return config_t<float, false>(v, blocks_per_sm, smem);
}

cudaError_t batch2d_launch(int prec, int v, const BatchArgs& b, int blocks, cudaStream_t s)
{
    if (prec == WENO_FP64) return launch_t<double, false>(v, b, blocks, s);
    if (prec == WENO_MIXED) return launch_t<float, true>(v, b, blocks, s);
    return launch_t<float, false>(v, b, blocks, s);
}

}  // namespace wis
