// Mixed instantiations: float storage and arithmetic, with the fifth
// difference of the detector (Eq. eq28), whose cancellation decides the
// hybrid switch, formed as exact nested float differences.
#include "weno_launch.cuh"

namespace wis {

cudaError_t sweep_mixed(int dim, int dir, int variant, const SweepArgs& a, cudaStream_t s)
{
    return launch_sweep_t<float, true>(dim, dir, variant, a, s);
}

}  // namespace wis
