// Mixed instantiations: float storage and bulk arithmetic; the fifth
// difference of the detector (Eq. eq28), whose cancellation decides the
// hybrid switch, is formed in double.
#include "weno_launch.cuh"

namespace wis {

cudaError_t sweep_mixed(int dim, int dir, const SweepArgs& a, cudaStream_t s)
{
    return launch_sweep_t<float, true>(dim, dir, a, s);
}

}  // namespace wis
