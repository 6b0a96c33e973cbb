// Internal types shared by the host runtime (ctx.cu) and the kernels of
// liblbm.so.  Nothing here is part of the C ABI (include/lbm.h).
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (types only; the encoder is fetched at run time)
#include <cuda_runtime.h>

#include "sweep_types.h"

namespace lbm {

// Ghost-exchange work item: one direction plane of one face or edge of a
// Block's ghost shell, a slab of `rows` rows of `len` contiguous elements
// (stride `stride` elements between rows), copied from the neighbour's
// matching boundary rows.  src / dst are element offsets into the buffer.
struct XSlab {
    long long src, dst;
    long long stride;
    int rows, len;
};
// A slab of the in-place scheme's reverse exchange: element (r, i) moves
// from src + r stride + i to dst + r stride + i when the flag at
// fsrc + r fstride + i (the cell that streamed it) is fluid.
struct XSlabF {
    long long src, dst;
    long long stride;
    long long fsrc, fstride;
    int rows, len;
};

// Sets the calling thread's message for lbm_last_error(NULL).
void set_global_error(const char *msg);

// cuTensorMapEncodeTiled from the driver (NULL when unavailable); cast to
// PFN_cuTensorMapEncodeTiled_v12000.
void *tma_encode_fn();

// The device allocator hooks in effect (lbm_set_allocator; NULL = cudaMalloc).
void current_allocator(void *(**alloc)(size_t, void *, void *), void (**release)(void *, size_t, void *, void *),
                       void **user);

// Reduction outputs per tile / instance.
enum { R_DRHO = 0, R_JX, R_JY, R_JZ, R_NFLUID, R_NONFINITE, R_DU2, R_U2, R_K };

// ---- launchers (kernels.cu / sweep.cu) ----

// TMA-staged sweep over a Patch whose Blocks all have nx = TX (32..256).
struct TmaSweepArgs {
    SweepArgs a;
    int nx, ny, nz;           // Block interior size (uniform)
    int px, py;               // PDF row pitch, rows per plane (uniform)
    int pxf;                  // flag row pitch
    int ngy;                  // row groups of TY rows per Block
    int zchunk, nzc;          // z slices per work item, work items along z per Block
    long long nitems;         // Blocks * ngy * nzc
    int parity;               // which tensor maps describe src
    int drop_stage;           // failure-path test: skip this stage's loads (-1 = none)
    long long wait_cycles;    // bound of every mbarrier wait
    int *err;                 // device error word (set on a timed-out wait)
};
// Tensor maps of the TMA sweep: the PDF buffers viewed as a 4-D tensor
// (x, y, z, 19 * Block + q), and the flag array as (x, y, z, Block).
struct TmaMaps {
    CUtensorMap box_a[2];  // per buffer: box {TX, TY, 1, 1} for directions with e_x = 0
    CUtensorMap box_b[2];  // {TX + A, TY, 1, 1} for e_x = +-1 (A = 16 bytes of elements)
    CUtensorMap halo[2];   // {A, TY, 1, 1}: boundary columns of the x-neighbour Blocks
    CUtensorMap flags;     // uint8 {TX, TY, 1, 1}
};
// Returns cudaErrorNotSupported when the Block width has no instantiation.
cudaError_t launch_sweep_tma(const TmaSweepArgs &a, const TmaMaps &maps, int grid, cudaStream_t s);
int tma_stages(int storage);
cudaError_t tma_occupancy(int storage, int tx, int collision, int forced, int *ctas_per_sm);
cudaError_t launch_sweep(const SweepArgs &a, cudaStream_t s);

struct ExchangeArgs {
    const XSlab *slabs;
    int nslabs;
    void *buf;
    int elem_bytes;
};
cudaError_t launch_exchange(const ExchangeArgs &a, cudaStream_t s);
cudaError_t launch_exchange_flagged(const XSlabF *slabs, int nslabs, void *buf, int elem_bytes,
                                    const uint8_t *flags, cudaStream_t s);
// Curved walls: clears L_CURVED on all nlinks masks, then validates the n
// links (flag index of the fluid cell, of its resting-wall source, table row)
// and sets idx / L_CURVED; *bad counts links whose kinds do not fit.
cudaError_t launch_curved_setup(const long long *fidx, const long long *sidx, const int *rows, long long n,
                                const uint8_t *flags, uint32_t *links, long long nlinks, int *idx, int *bad,
                                cudaStream_t s);
// The sweep over the fluid-cell list (sweep_sparse.cu).
cudaError_t launch_sweep_sparse(const SweepArgs &a, cudaStream_t s);
// In-place (AA-pattern) sweep: mode 0 even step, 1 odd step, 2 gather of an
// odd-time state into the natural layout of a.dst.
cudaError_t launch_sweep_aa(const SweepArgs &a, int mode, cudaStream_t s);

struct FieldArgs {
    const Tile *tiles;
    long long ntiles;
    const BlockGeom *blocks;
    const void *consts;
    const uint8_t *flags;
    int tx, ty, tz;
    int storage;
    int swap;  // 1: direction q of a cell is stored in slot opp(q) (the in-place
               // scheme at an even time)
    const int *sidx;     // fluid-cell list layout: list index per flag cell (-1 solid), else NULL
    long long sstride;   // its direction stride
};
// rho/u in the concatenated output layout (device pointers)
cudaError_t launch_macroscopic(const FieldArgs &a, const void *buf, float *rho, float *u,
                               cudaStream_t s);
cudaError_t launch_init_equilibrium(const FieldArgs &a, void *buf, const float *rho,
                                    const float *u, cudaStream_t s);
// f64 <-> storage, concatenated PDF layout
cudaError_t launch_get_pdfs(const FieldArgs &a, const void *buf, double *f, cudaStream_t s);
cudaError_t launch_set_pdfs(const FieldArgs &a, void *buf, const double *f, cudaStream_t s);
cudaError_t launch_zero(void *buf, size_t bytes, cudaStream_t s);
// Sets the velocity of every fluid cell to u (macroscopic layout), keeping
// density and the non-equilibrium part
cudaError_t launch_impose_velocity(const FieldArgs &a, void *buf, const float *u, cudaStream_t s);
// Velocity change against a stored velocity field (macroscopic layout)
cudaError_t launch_reduce_snap(const FieldArgs &a, const void *cur, const float *usnap, double *partial,
                               const long long *inst_tile_begin, int ninst, double *out, cudaStream_t s);
// FP64 reductions: per-tile partials then per-instance totals
cudaError_t launch_reduce(const FieldArgs &a, const void *cur, const void *prev, double *partial,
                          const long long *inst_tile_begin, int ninst, double *out,
                          cudaStream_t s);

}  // namespace lbm
