// staged.cuh -- host/device interface of the shared-memory-staged B-spline evaluation
// (eval_staged.cu) and of the pencil order it reads (order.cu).
#pragma once

#include <cuda.h>   // CUtensorMap (the descriptor type only; no driver library is linked)

#include "qmcspl_internal.cuh"

namespace qmcspl {

constexpr int kBox = 5;                       // (x, y) columns per pencil axis: 2 cells + 3 stencil overhang
constexpr int kPlaneRows = kBox * kBox;       // rows of one staged z plane, per table
constexpr int kPencilEdge = 2;                // grid cells per pencil edge in x and y
#ifndef QMCSPL_STAGED_CONSUMERS
#define QMCSPL_STAGED_CONSUMERS 8
#endif
constexpr int kStagedConsumers = QMCSPL_STAGED_CONSUMERS;   // consumer warps per block (plus one producer warp)
constexpr int kStagedRingOffset = 1024;       // barriers and flags before the plane ring
constexpr int kStagedMaxSmem = 227 * 1024;    // dynamic shared memory of one block
constexpr int kStagedMaxSlots = 16;
constexpr int kStagedMinSlots = 6;            // 4 planes per position + 2 in flight
constexpr long long kMaxPencilBins = 1LL << 22;
// Tensor maps per table, one per box shape: kBox y rows by 1..5 x rows (index bx - 1), and one
// x row by 1..4 y rows (index kBox + by - 1) for boxes that wrap around the cell in y.
constexpr int kStagedMaps = 9;

struct StagedMaps {
    CUtensorMap m[2][kStagedMaps];   // [table][box shape], 4-D view [x][y][z][orbital] of the table
};

struct StagedArgs {
    const int* bin_end;       // after the counting sort: one past the last position of every bin
    int npx, npy;             // pencils per axis
    int zseg, nseg;           // z cells per work item, work items per pencil
    long long n_items;        // pencils x nseg
    int slots;                // plane slots in the ring
    int row_bytes;            // bytes of one stored row (O_p x element size)
    int n_tab;                // tables staged: 1, or 2 with the separate Laplacian table
    int elem_bytes;
    int stall;                // test hook: the producer copies nothing (qmcspl_debug_stall_pipeline)
};

inline size_t staged_smem_bytes(const StagedArgs& s)
{
    return kStagedRingOffset + (size_t)s.slots * s.n_tab * kPlaneRows * s.row_bytes;
}

// True when the handle's evaluation can run staged: cubic B-splines on a uniform grid
// without separate gradient tables, FP32 or BF16 tables, one orbital tile per position, rows
// of 128, 256 or 512 bytes, a plane ring of at least kStagedMinSlots slots in shared memory,
// and a driver that encodes tensor maps.
bool staged_eligible(const Handle* h);
// Pencil-order bin geometry (bins of 2 x 2 x 1 cells) and the staged launch shape of a handle
// for n_pos positions; false if the bins would be too many.
bool staged_plan(const Handle* h, long long n_pos, BinGeometry* g, StagedArgs* s);
// True when qmcspl_eval_vgl of n_pos positions should sort them into pencils and run staged:
// eligible handles in QMCSPL_ORDER_PENCIL (never chosen automatically).
bool use_staged(const Handle* h, long long n_pos);
// Evaluate positions prepared in the pencil order of staged_plan (records, permutation and
// bin ends in `pr`).
int launch_bspline_vgl_staged(const Handle* h, const Prepared& pr, long long n_pos, void* val, void* grad,
                              void* lap, StagedArgs s, cudaStream_t stream);

}  // namespace qmcspl
