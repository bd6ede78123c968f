// vb_colour_meas.cu -- instantiations of the packed VB sweep that also measure the energy
// (Eq. 3) of the state the sweep starts from; see vb_colour.cuh.
#include "vb_colour.cuh"

namespace sg {

int vb_packed_sweep_meas(const VbPackedDev& d, const uint32_t* colour_groups,
                         const uint32_t* clock, uint32_t t_off, int variant, bool fused,
                         const VbSweepMeas& meas, cudaStream_t st) {
    return packed_sweep<true>(d, colour_groups, clock, t_off, variant, fused, meas, st);
}

}  // namespace sg
