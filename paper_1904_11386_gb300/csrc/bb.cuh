// Bounce-back launches split for the step, whose list reset and mass bookkeeping can run beside other kernels.
#pragma once

#include "scbb_internal.cuh"

namespace scbb {

// Clears the previous step's boundary and fresh bits and the column counters; saves the previous step's
// fresh-node count for the mass bookkeeping.
void launch_bb_lists_reset(const DevState& d, cudaStream_t st);
// Classification at the current positions and the boundary list with crossed elements (after the reset):
// launch_bb_owner (column lists, owner field, fresh list) then launch_bb_boundary_list (boundary list and
// crossed elements), which reads nothing the fresh-node kernels write.
void launch_bb_classify_lists(const LbmParams& p, const DevState& d, int step, bool init, cudaStream_t st);
void launch_bb_owner(const LbmParams& p, const DevState& d, int step, bool init, cudaStream_t st);
void launch_bb_boundary_list(const LbmParams& p, const DevState& d, cudaStream_t st);
constexpr int BB_LIST_LAUNCHES = 3;     // kernels of launch_bb_boundary_list
// Settles the crossed element of every cut link of the current boundary list (and the virtual densities the
// boundary kernel reads); the first kernel of the step's boundary phase.
void launch_bb_vrho(const LbmParams& p, const DevState& d, cudaStream_t st);
// Mass bookkeeping and correction factors of Eq. 18 (after this step's boundary kernel).
void launch_bb_mass(const LbmParams& p, const DevState& d, cudaStream_t st);
// New populations of the fresh nodes (after the classification and the mass bookkeeping).
void launch_bb_fresh_nodes(const LbmParams& p, const DevState& d, float* Snew, int step, cudaStream_t st);

}  // namespace scbb
