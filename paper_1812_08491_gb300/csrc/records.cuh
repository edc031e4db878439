// records.cuh -- SepSet record groups of a single call's pool and the
// launchers of the device-built result lists (k_records.cu).
#pragma once

#include <cuda_runtime.h>

#include "cupc.h"

namespace cupc {

// SepSet records of removals at levels >= 1 in a single call's pool, grouped
// by level: level lev[q] has count[q] records of 3 + lev[q] ints (i, j, l, S)
// starting at int start[q]; first[q] is the index of its first record over all
// groups, total the number of records.
constexpr int kRecGroups = CUPC_MAX_LEVEL + 1;
struct RecGroups {
    int groups;
    int lev[kRecGroups];
    long long start[kRecGroups];
    long long count[kRecGroups];
    long long first[kRecGroups];
    long long total;
};

struct ProbDesc;

// Rows the list builders walk: one problem (vprob == nullptr: W words a row,
// p columns), or a batch's block-diagonal union (row g belongs to problem
// vprob[g], whose bitset block holds its local columns).
struct RowView {
    const int* vprob;
    const ProbDesc* probs;
    int W, p;
};

// The records in (i, j) order, ids local to their problem, into out (all the
// pool's ints) and, in status[0..2], the bit flags of a failed check, the
// number of removed pairs (bits of bits0 & ~bits with j > i) and the ints
// placed; rowoff[g] = the int offset of row g's records. Batches also count
// the records per problem and level into plc (zeroed; plc_stride per
// problem). Scratch: wpre one word per bitset word, rowcnt and rowints nrows,
// rowstart and rowoff nrows + 1, slot G.total.
cudaError_t launch_records_sort(const int* rec, const RecGroups& G, const unsigned* bits, const unsigned* bits0,
                                const RowView& V, long long nrows, unsigned* wpre, long long* rowcnt,
                                long long* rowstart, unsigned long long* rowints, long long* rowoff, long long* slot,
                                int* out, long long* status, unsigned long long* plc, int plc_stride, cudaStream_t st);
// The edge list: pairs i < j of bits in (i, j) order, at most cap pairs into
// out; status[0] = the number of edges. Scratch: rowcnt p, off p + 1.
cudaError_t launch_edge_list(const unsigned* bits, int p, int W, long long* rowcnt, long long* off, long long cap,
                             int* out, long long* status, cudaStream_t st);

}  // namespace cupc
