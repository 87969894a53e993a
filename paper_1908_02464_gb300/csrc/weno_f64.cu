// FP64 instantiations: all arithmetic and storage in double.
#include "weno_launch.cuh"

namespace wis {

cudaError_t sweep_f64(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s)
{
    return launch_sweep_t<double, false>(dim, dir, variant, a, s);
}
cudaError_t cfl_f64(int dim, const CflArgs& a, int nsm, cudaStream_t s) { return launch_cfl_t<double>(dim, a, nsm, s); }
cudaError_t totals_f64(int dim, const TotArgs& a, int blocks, cudaStream_t s)
{
    return launch_totals_t<double>(dim, a, blocks, s);
}
cudaError_t pack_f64(const void* src, void* dst, int nv, const int* n, long long sy, long long sz, long long sv,
                     long long off0, int to_ghosted, int nsm, cudaStream_t s)
{
    return launch_pack_t<double>(src, dst, nv, n, sy, sz, sv, off0, to_ghosted, nsm, s);
}

cudaError_t vjp_f64(int dim, int dir, const VjpArgs& a, cudaStream_t s)
{
    return launch_vjp_t<double>(dim, dir, a, s);
}
long long vjp_tiles_f64(int dim, int dir, const int* n) { return vjp_tiles_t<double>(dim, dir, n); }
cudaError_t ghost_adj_f64(int dim, const GhostArgs& a, const void* ghost, void* G, cudaStream_t s)
{
    return launch_ghost_adj_t<double>(dim, a, ghost, G, s);
}

cudaError_t lf_f64(int dim, const CflArgs& a, unsigned long long* out, int nsm, cudaStream_t s)
{
    return launch_lf_t<double>(dim, a, out, nsm, s);
}

}  // namespace wis
