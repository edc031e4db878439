// orient.cuh -- launchers of the orientation kernels (k_orient.cu): the second
// step of PC-stable (Sec. 2.4), v-structures and Meek's rules on bitsets.
#pragma once

#include <cuda_runtime.h>

#include "cupc.h"
#include "records.cuh"

namespace cupc {

// SepSet records of removals at levels >= 1, grouped by level (RecGroups).
using OrRecords = RecGroups;

// Neighbour lists of the skeleton bitset: deg, exclusive offsets off[0..p], cols.
cudaError_t launch_or_degree(const unsigned* bits, int p, int W, int* deg, cudaStream_t st);
cudaError_t launch_or_scan(const int* deg, int p, long long* off, cudaStream_t st);
cudaError_t launch_or_fill(const unsigned* bits, int p, int W, const long long* off, int* cols, cudaStream_t st);
// v-structures i -> k <- j: pairs removed at level 0 (S empty; bits0 = A_G after
// level 0) and pairs with a SepSet record
cudaError_t launch_or_vstruct0(const unsigned* bits, const unsigned* bits0, int p, int W, const long long* off,
                               const int* cols, unsigned* head, unsigned* headT, cudaStream_t st);
cudaError_t launch_or_vstructS(const unsigned* bits, int p, int W, const long long* off, const int* cols,
                               const int* rec, const OrRecords& R, unsigned* head, unsigned* headT, cudaStream_t st);
// one round of Meek's rules: proposals from the round's starting marks, then
// their application; flags[0] += orientations applied, flags[1] += pairs
// proposed both ways (each counted from both ends). With a gate (the previous
// round's flags[0]) both launches do nothing when that round applied nothing,
// so several rounds can be queued before the host looks.
cudaError_t launch_or_propose(const unsigned* bits, int p, int W, const long long* off, const int* cols,
                              const unsigned* head, const unsigned* headT, unsigned* prop,
                              const unsigned long long* gate, cudaStream_t st);
cudaError_t launch_or_apply(const unsigned* prop, int p, int W, unsigned* head, unsigned* headT,
                            unsigned long long* flags, const unsigned long long* gate, cudaStream_t st);
// p x p edge marks (0 none, 1 arrowhead at the column's end, 2 tail) and the
// counts flags[2..4] += directed, undirected, bidirected edges
cudaError_t launch_or_marks(const unsigned* bits, const unsigned* headT, int p, int W, unsigned char* marks,
                            unsigned long long* flags, cudaStream_t st);

}  // namespace cupc
