// Membrane launches split for the bounce-back step, whose elastic part can run beside the fluid kernels.
#pragma once

#include "scbb_internal.cuh"

namespace scbb {

// Forces that depend on the vertex positions alone: particle-particle repulsion (Eq. 26), the Skalak and
// bending passes and the capsule reduction (volume, centre, classification box).  Returns the launch count.
int launch_membrane_elastic(const LbmParams& p, const DevState& d, cudaStream_t st);

// Adds the bounce-back coupling (bb) or nothing, and moves the vertices (forward Euler).  Returns the launch
// count.
int launch_membrane_update(const LbmParams& p, const DevState& d, bool bb, int step, cudaStream_t st);

}  // namespace scbb
