// FP32 instantiations: float storage and arithmetic (the CFL max, the time
// step, the time and the conserved totals stay in double).
#include "weno_launch.cuh"

namespace wis {

cudaError_t sweep_f32(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s)
{
    return launch_sweep_t<float, false>(dim, dir, variant, a, s);
}
cudaError_t cfl_f32(int dim, const CflArgs& a, int nsm, cudaStream_t s) { return launch_cfl_t<float>(dim, a, nsm, s); }
cudaError_t totals_f32(int dim, const TotArgs& a, int blocks, cudaStream_t s)
{
    return launch_totals_t<float>(dim, a, blocks, s);
}
cudaError_t pack_f32(const void* src, void* dst, int nv, const int* n, long long sy, long long sz, long long sv,
                     long long off0, int to_ghosted, int nsm, cudaStream_t s)
{
    return launch_pack_t<float>(src, dst, nv, n, sy, sz, sv, off0, to_ghosted, nsm, s);
}

cudaError_t vjp_f32(int dim, int dir, const VjpArgs& a, cudaStream_t s)
{
    return launch_vjp_t<float>(dim, dir, a, s);
}
long long vjp_tiles_f32(int dim, int dir, const int* n) { return vjp_tiles_t<float>(dim, dir, n); }
cudaError_t ghost_adj_f32(int dim, const GhostArgs& a, const void* ghost, void* G, cudaStream_t s)
{
    return launch_ghost_adj_t<float>(dim, a, ghost, G, s);
}

cudaError_t lf_f32(int dim, const CflArgs& a, unsigned long long* out, int nsm, cudaStream_t s)
{
    return launch_lf_t<float>(dim, a, out, nsm, s);
}

}  // namespace wis
