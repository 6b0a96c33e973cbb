// Internal types shared by the host runtime (ctx.cu) and the kernels of
// liblbm.so.  Nothing here is part of the C ABI (include/lbm.h).
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap (types only; the encoder is fetched at run time)
#include <cuda_runtime.h>

namespace lbm {

constexpr int Q = 19;

// D3Q19 velocity components packed two bits per direction (value + 1), in the
// order documented in include/lbm.h.  constexpr so that fully unrolled kernel
// loops fold every e_q component into an immediate.
__host__ __device__ constexpr int ex(int q) { return int((0x1548889549ull >> (2 * q)) & 3u) - 1; }
__host__ __device__ constexpr int ey(int q) { return int((0x895609495ull >> (2 * q)) & 3u) - 1; }
__host__ __device__ constexpr int ez(int q) { return int((0x20a0954955ull >> (2 * q)) & 3u) - 1; }
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
// Lattice weights of Sec. 2.1: 1/3 rest, 1/18 axis, 1/36 diagonal.
__host__ __device__ constexpr int norm2(int q) { return ex(q) * ex(q) + ey(q) * ey(q) + ez(q) * ez(q); }
__host__ __device__ constexpr double wq(int q) { return norm2(q) == 0 ? 1.0 / 3.0 : (norm2(q) == 1 ? 1.0 / 18.0 : 1.0 / 36.0); }

// Internal flag byte of a stored cell (interior or ghost).
enum : uint8_t {
    F_FLUID = 0,
    F_NOSLIP = 1,
    F_MOVING = 2,
    F_KIND = 3,   // mask of the kind bits
    F_NEAR = 4,   // fluid cell with at least one wall / solid neighbour
};

// Stored x index of the first interior cell of every row: 16 cells, so that
// interior rows start on a 32-byte DRAM sector for every PDF type and the
// one-byte flag rows start 16-byte aligned (a TMA requirement).
constexpr int OX = 16;

// One Block (or one batch instance) in device memory.  The Block stores
// (nx+2)(ny+2)(nz+2) logical cells with x padded: row pitch px (a multiple of
// 16 cells), the first interior cell of a row at x index ox = OX, ghost cells
// at ox-1 and ox+nx.  PDF plane q of the Block
// lives at buf + pdf_base + q*G, flag byte of cell c at flags + cell_base + c.
//
// Across x faces the sweep reads the neighbouring Block's boundary column
// directly (xm_off / xp_off: element offset from this Block's stored cell
// x = ox-1 / ox+nx to the matching interior cell of the -x / +x neighbour,
// 0 where the face is a wall), so the ghost exchange copies only the y and z
// faces and the yz edges, which are contiguous rows in this layout.
struct BlockGeom {
    long long pdf_base;   // elements
    long long cell_base;  // cells (flags)
    long long G;          // cells per plane = px*py*pz
    long long xm_off, xp_off;
    // Fused ghost writes: element offset from this Block's stored cell to the
    // ghost cell of the neighbour that pulls it, for the -y, +y, -z, +z faces
    // and the (-y,-z), (+y,-z), (-y,+z), (+y,+z) edges; bit k of push_mask is
    // set when neighbour k exists.
    long long push_off[8];
    int push_mask;
    int xm_block, xp_block;  // -x / +x neighbour Block, -1 where the face is a wall
    int nx, ny, nz;       // interior cells
    int px, py;           // padded row pitch (cells), rows per plane (ny+2)
    int ox;               // x index of the first interior cell
    int inst;             // instance this block belongs to
    int gx, gy, gz;       // origin of the block inside its instance
    long long out_base;   // first cell of the instance in the concatenated output
    int NX, NY, NZ;       // instance size
    int pad_;
};

// Collision constants of one instance in scaled units (scale s of the
// storage; s = 1 for F32 / F64):
//   drho_s = sum g,   u = (sum e g) * ufac + uoff  with ufac = 1/(s rho0), uoff = F/(2 rho0)
//   feq_s  = w (drho_s + rho0s (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)),  rho0s = s rho0
//   Guo source (scaled): cp w (9 (e.u)(e.Fs) - 3 u.Fs) + cm w 3 (e.Fs),  Fs = s F
template <typename T>
struct CollideConsts {
    T rho0s, ufac, uoff[3];
    T omega_p, omega_m, cp, cm;
    T Fs[3];
    T bbw[Q];     // s * 6 w_q rho0 (e_q . u_wall)
    T inv_s, rho0;
};

// Sweep work item: one CTA updates tx*ty*tz cells starting at (x0,y0,z0)
// of block `block` (interior coordinates).
struct Tile {
    int block, x0, y0, z0;
};

// Ghost-exchange work item: copy, for every cell of a region of the ghost
// shell of dst_block, the listed directions from the interior of src_block.
struct XDesc {
    int dst_block, src_block;
    int x0, y0, z0;        // region start in interior coordinates (-1 or n for the ghost side)
    int lx, ly, lz;        // region extent
    int sx, sy, sz;        // source cell = region cell + (sx,sy,sz)
    int ndir;
    int dir[5];
    int ncell;             // lx*ly*lz
};

// Sets the calling thread's message for lbm_last_error(NULL).
void set_global_error(const char *msg);

// Reduction outputs per tile / instance.
enum { R_DRHO = 0, R_JX, R_JY, R_JZ, R_NFLUID, R_NONFINITE, R_DU2, R_U2, R_K };

// ---- launchers (kernels.cu / sweep.cu) ----
struct SweepArgs {
    const Tile *tiles;
    long long ntiles;
    const BlockGeom *blocks;
    const void *consts;       // CollideConsts<T>[instances], T = double for F64 else float
    const uint8_t *flags;
    const void *src;
    void *dst;
    int tx, ty, tz;
    int collision;            // 0 BGK, 1 TRT
    int forced;               // any instance has a nonzero force
    int storage;              // LBM_F32 .. LBM_F64
    int grid;                 // CTAs to launch (<= ntiles; persistent loop when smaller)
    int minb;                 // register budget: 3 or 4 resident 256-thread CTAs per SM
    int push;                 // 1: write boundary PDFs into the neighbours' ghost layers
};

// TMA-staged sweep over a Patch whose Blocks all have nx = TX (32..256).
struct TmaSweepArgs {
    SweepArgs a;
    int nx, ny, nz;           // Block interior size (uniform)
    int px, py;               // stored pitch (uniform)
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

// Exchange CTA work list: CTA k copies items [first, first + blockDim) of
// descriptor desc (items are direction-major, x fastest within a direction).
struct XWork {
    int desc;
    int first;
};
struct ExchangeArgs {
    const XDesc *desc;
    const XWork *work;
    int nwork;
    const BlockGeom *blocks;
    void *buf;
    int elem_bytes;
};
cudaError_t launch_exchange(const ExchangeArgs &a, cudaStream_t s);

struct FieldArgs {
    const Tile *tiles;
    long long ntiles;
    const BlockGeom *blocks;
    const void *consts;
    const uint8_t *flags;
    int tx, ty, tz;
    int storage;
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
// FP64 reductions: per-tile partials then per-instance totals
cudaError_t launch_reduce(const FieldArgs &a, const void *cur, const void *prev, double *partial,
                          const long long *inst_tile_begin, int ninst, double *out,
                          cudaStream_t s);

}  // namespace lbm
