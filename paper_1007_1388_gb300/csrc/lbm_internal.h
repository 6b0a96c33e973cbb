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

// Link mask of a fluid cell with F_NEAR set (one uint32 per flag cell, same
// indexing as the flags): bit q (1..18) is set when the pull source x - e_q is
// a wall or solid cell, so that g_q comes from half-way bounce-back; bit
// L_MOVING when at least one of those sources is a moving wall.
constexpr uint32_t L_MOVING = 1u << 31;

// Layout of a Block.  PDF planes store (ny+2)(nz+2) rows of px cells: the
// interior x range [0, nx) padded only up to a 32-byte multiple, plus one ghost
// row on each y and z side.  There are no x ghost columns: across x faces the
// sweep reads the neighbouring Block's boundary column directly, so a row is
// exactly the data the sweep needs and the L2's 64-256-byte fetches carry no
// padding.  The flag array keeps one ghost cell on every side (its interior x
// starts at OXF = 16 so that flag rows are 16-byte aligned for TMA).
constexpr int OXF = 16;

// PDF of cell (x,y,z) in direction q: buf[pdf_base + q*G + c] with
// c = ((z+1)*py + y+1)*px + x; its flag: flags[cell_base + cf] with
// cf = ((z+1)*py + y+1)*pxf + x + OXF.  xm_off / xp_off: element offset that
// moves a pull across the -x / +x face into the neighbouring Block (0 where
// the face is a wall; the flags then make the pull a bounce-back).
struct BlockGeom {
    long long pdf_base;   // elements
    long long cell_base;  // flag bytes
    long long G;          // PDF cells per plane = px*py*(nz+2)
    long long Gf;         // flag cells = pxf*py*(nz+2)
    long long xm_off, xp_off;
    int xm_block, xp_block;  // -x / +x neighbour Block, -1 where the face is a wall
    int nx, ny, nz;       // interior cells
    int px, py;           // PDF row pitch (cells), rows per plane (ny+2)
    int pxf;              // flag row pitch (cells)
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
// Per-instance constants.  The first group serves the moment, conversion
// and bounce-back kernels; the second the collision (collide.cuh), with the
// Guo source folded into the equilibrium and the relaxation rates folded into
// the coefficients:  a+ = (1 - omega+/2)/omega+,  a- = (1 - omega-/2)/omega-,
// w_c = 1/18 (axis pairs, c = 0) or 1/36 (diagonal pairs, c = 1), and
// omega = omega+ = omega- for BGK.
template <typename T>
struct CollideConsts {
    T rho0s, ufac, uoff[3];   // rho0s = s rho0; u = j ufac + uoff, ufac = 1/(s rho0), uoff = F/(2 rho0)
    T omega_p, omega_m;
    T Fs[3];                  // s F
    T bbw[Q];                 // s * 6 w_q rho0 (e_q . u_wall)
    T inv_s, rho0;
    T zero;                   // 0
    T nc15, c45;              // -1.5 rho0s, 4.5 rho0s
    T k9F[3], nk3F[3];        // 9 a+ Fs, -3 a+ Fs
    T c0a, c0b;               // omega+ / 3, 1 - omega+
    T obw[2], oc3[2];         // BGK: omega w_c, omega 3 rho0s w_c
    T okF[2][3];              // BGK: omega 3 a- w_c Fs
    T hwp, hwm;               // TRT: omega+/2, omega-/2
    T nwpw[2], nwmc3[2];      // TRT: -omega+ w_c, -omega- 3 rho0s w_c
    T nwmkF[2][3];            // TRT: -omega- 3 a- w_c Fs
};

// Sweep work item: one CTA updates tx*ty*tz cells starting at (x0,y0,z0)
// of block `block` (interior coordinates).  In the flat sweep a tile is the
// run of tx cells of the Block starting at linear index x0 = (z ny + y) nx + x.
struct Tile {
    int block, x0, y0, z0;
};

// Ghost-exchange work item: one direction plane of one face or edge of a
// Block's ghost shell, a slab of `rows` rows of `len` contiguous elements
// (stride `stride` elements between rows), copied from the neighbour's
// matching boundary rows.  src / dst are element offsets into the buffer.
struct XSlab {
    long long src, dst;
    long long stride;
    int rows, len;
};

// Sets the calling thread's message for lbm_last_error(NULL).
void set_global_error(const char *msg);

// The device allocator hooks in effect (lbm_set_allocator; NULL = cudaMalloc).
void current_allocator(void *(**alloc)(size_t, void *, void *), void (**release)(void *, size_t, void *, void *),
                       void **user);

// Reduction outputs per tile / instance.
enum { R_DRHO = 0, R_JX, R_JY, R_JZ, R_NFLUID, R_NONFINITE, R_DU2, R_U2, R_K };

// ---- launchers (kernels.cu / sweep.cu) ----
struct SweepArgs {
    const Tile *tiles;
    long long ntiles;
    const BlockGeom *blocks;
    const void *consts;       // CollideConsts<T>[instances], T = double for F64 else float
    const uint8_t *flags;
    const uint32_t *links;    // link masks of near-wall cells (flag indexing)
    const void *src;
    void *dst;
    int tx, ty, tz;
    int flat;                 // 1: a tile is a run of tx consecutive cells of a Block in
                              // (z, y, x) order starting at linear cell index x0
    int mask;                 // 1: near-wall cells via link masks under a warp vote
    int collision;            // 0 BGK, 1 TRT
    int forced;               // any instance has a nonzero force
    int storage;              // LBM_F32 .. LBM_F64
    int grid;                 // CTAs to launch (<= ntiles; persistent loop when smaller)
    int minb;                 // register budget: 3 or 4 resident 256-thread CTAs per SM
    int unif;                 // 1: a single instance, whose constants are kf (FP32
                              // arithmetic) or kd (FP64) and reach the kernel as parameters
    CollideConsts<float> kf;
    CollideConsts<double> kd;
};

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
