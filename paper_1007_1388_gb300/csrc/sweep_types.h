// Types and constants that define the fused sweep kernel: the D3Q19 table,
// the flag bits, the Block layout, the collision constants, the work items and
// the sweep's launch arguments.  Internal to liblbm.so (not part of the C ABI).
#pragma once

#include <cstdint>
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
    F_PRESSURE = 3,  // pressure boundary (anti-bounce-back to density rho_b)
    F_KIND = 3,   // mask of the kind bits
    F_NEAR = 4,   // fluid cell with at least one wall / solid neighbour
    F_FILL = 8,   // FP32/16-bit: interior no-slip cell sharing a 32-byte PDF sector with a fluid cell
    F_PAD = 16,   // FP32: cell nx - 1 - j of a row (j in the bits above) also zeroes padding element nx + j
};
constexpr int F_PAD_SHIFT = 5;  // j < 8: a row of 32-byte sectors has at most 7 FP32 padding elements

// Link mask of a fluid cell with F_NEAR set (one uint32 per flag cell, same
// indexing as the flags): bit q (1..18) is set when the pull source x - e_q is
// a wall or solid cell, so that g_q comes from half-way bounce-back; bit
// L_MOVING when at least one of those sources is a moving wall, L_PRESSURE
// when one is a pressure boundary.
constexpr uint32_t L_MOVING = 1u << 31;
constexpr uint32_t L_PRESSURE = 1u << 30;
// some pull of the cell crosses a curved resting wall (its distances are in
// the curved-link table)
constexpr uint32_t L_CURVED = 1u << 29;

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
    // n / nx and n / ny for 0 <= n < 2^31 as (n * m) >> sh (div_magic, quot)
    uint32_t mnx, mny;
    int snx, sny;
    // in-place streaming: side storage of the slots of the cells just beyond
    // a wall -x / +x face (what the pull-and-push step streams into the wall,
    // and pressure nodes' prepared values); element offset in the PDF buffer
    // of [5 directions with e_x = -1 / +1][py * (nz + 2) rows], -1 where the
    // face has a neighbour Block (or two arrays are used)
    long long xw_base[2];
};

// Division by a run-time divisor d >= 1 as a multiply and a shift (the
// multiply-shift method of Granlund and Montgomery, "Division by invariant
// integers using multiplication", 1994): with 2^s >= d and
// m = ceil(2^(31+s) / d) < 2^32, floor(n m / 2^(31+s)) = floor(n / d) for every
// 0 <= n < 2^31, because n m / 2^(31+s) exceeds n / d by less than 2^-s <= 1/d.
inline void div_magic(uint32_t d, uint32_t *m, int *sh)
{
    int s = 0;
    while ((1ull << s) < d) ++s;
    *m = uint32_t(((1ull << (31 + s)) + d - 1) / d);
    *sh = 31 + s;
}
__host__ __device__ __forceinline__ int quot(int n, uint32_t m, int sh)
{
    return int((unsigned long long)(unsigned)n * m >> sh);
}

// index 0..4 of direction q among the five with the same e_x (ascending q)
__host__ __device__ constexpr int xdir_index(int q)
{
    int k = 0;
    for (int r = 0; r < q; ++r) k += ex(r) == ex(q) ? 1 : 0;
    return k;
}

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
    int pair;                 // 1: two neighbouring cells (x even, x + 1) per thread; tx threads
                              // cover 2 tx cells (a flat tile: 2 tx consecutive cells)
    int collision;            // 0 BGK, 1 TRT
    int forced;               // any instance has a nonzero force
    int storage;              // LBM_F32 .. LBM_F64
    int grid;                 // CTAs to launch (<= ntiles; persistent loop when smaller)
    int minb;                 // register budget: 3, 4 or 5 resident 256-thread CTAs per SM
    int unif;                 // 1: a single instance, whose constants are kf (FP32
                              // arithmetic) or kd (FP64) and reach the kernel as parameters
    CollideConsts<float> kf;
    CollideConsts<double> kd;
    // pressure boundaries: 2 s (rho_b - rho0) (one value per context); the
    // anti-bounce-back term of direction q is w_q times this
    float pbf;
    double pbd;
    int pres;                 // bit 0: the Patch has pressure boundaries, bit 1: curved walls
                              // (each selects kernels built for it)
    // curved walls: per flag cell the row of the link table (-1: none), and
    // the table, 18 wall distances per row (directions 1..18) in the
    // arithmetic type; 1/2 on links that are half-way bounce-back
    const int *curv_idx;
    const void *curv_q;
    // fluid-cell list layout: neighbour table [19][nstride] (row 0: bit 0 =
    // the cell has a pressure link; rows 1..18: the pull source's list index,
    // or -1 resting wall, -2 moving wall, -3 pressure node), fluid cells, and
    // the stride of the PDF and neighbour rows
    const int *nbr;
    long long nfluid, nstride;
};

}  // namespace lbm
