// The context builder of the host runtime: the Block layout of a Patch or a
// batch (row pitch, plane size, ghost shell, x-face offsets), the flag field
// and the near-wall link masks, the ghost-exchange plans (two arrays and in
// place), the fluid-cell list's numbering and neighbour table, the sweep's
// work lists and the TMA sweep's tensor maps.
#include "ctx_internal.h"
#include "sector_fill.h"

using namespace lbm;

namespace lbm {
namespace rt {

int round_up(int v, int a) { return (v + a - 1) / a * a; }

// Cells per PDF plane: the stored cells padded so that the plane stride in
// bytes is an odd multiple of `unit` bytes.  The 19 read and 19 write streams
// of a sweep are one plane apart; a stride with a large power-of-two factor
// lines them up on the same DRAM channels.
long long plane_cells(long long cells, int elem)
{
    const long long unit = 256;
    const long long per = std::max<long long>(unit / elem, 16);
    long long k = (cells + per - 1) / per;
    if ((k & 1) == 0) ++k;
    return k * per;
}

// What lies at instance position (X,Y,Z): periodic axes wrap; beyond one
// non-periodic face is that face's wall; beyond two or more (an edge or
// corner of the wall shell) is a resting wall.
uint8_t classify(const lbm_params &p, const int N[3], const uint8_t *flags, long long X, long long Y,
                 long long Z)
{
    long long pos[3] = {X, Y, Z};
    int beyond = 0, face = 0;
    for (int a = 0; a < 3; ++a) {
        if (pos[a] >= 0 && pos[a] < N[a]) continue;
        if (p.periodic[a]) {
            pos[a] = ((pos[a] % N[a]) + N[a]) % N[a];
        } else {
            ++beyond;
            face = 2 * a + (pos[a] < 0 ? 0 : 1);
        }
    }
    if (beyond >= 2) return F_NOSLIP;
    if (beyond == 1) return uint8_t(p.face_bc[face]);
    if (!flags) return F_FLUID;
    return flags[(pos[2] * N[1] + pos[1]) * N[0] + pos[0]];
}

void build_tiles(lbm_ctx *c, const int t[3], std::vector<Tile> &tiles, std::vector<long long> &begin)
{
    tiles.clear();
    begin.assign(c->ninst + 1, 0);
    int inst = -1;
    for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
        const BlockGeom &b = c->blocks[bi];
        while (inst < b.inst) begin[++inst] = (long long)tiles.size();
        for (int z = 0; z < b.nz; z += t[2])
            for (int y = 0; y < b.ny; y += t[1])
                for (int x = 0; x < b.nx; x += t[0]) tiles.push_back({int(bi), x, y, z});
    }
    while (inst < c->ninst) begin[++inst] = (long long)tiles.size();
}


int validate_params(const lbm_params &p)
{
    if (p.collision != LBM_BGK && p.collision != LBM_TRT) return 0;
    if (p.storage < LBM_F32 || p.storage > LBM_F64) return 0;
    if (!(p.rho0 > 0) || !std::isfinite(p.rho0)) return 0;
    if (p.collision == LBM_TRT && !(p.magic > 0)) return 0;
    for (int f = 0; f < 6; ++f)
        if (p.face_bc[f] != LBM_NOSLIP && p.face_bc[f] != LBM_MOVING && p.face_bc[f] != LBM_PRESSURE) return 0;
    if (!(p.rho_b >= 0) || !std::isfinite(p.rho_b)) return 0;  // 0 = rho0
    double s = p.storage_scale;
    if (p.kernel < LBM_KERNEL_AUTO || p.kernel > LBM_KERNEL_TMA) return 0;
    if (p.streaming != LBM_STREAM_TWO_GRID && p.streaming != LBM_STREAM_AA) return 0;
    if (p.layout != LBM_LAYOUT_BLOCKS && p.layout != LBM_LAYOUT_SPARSE) return 0;
    int e2 = 0;
    if (!(s > 0) || !std::isfinite(s) || std::frexp(s, &e2) != 0.5) return 0;  // power of two
    return 1;
}

template <typename T>
std::vector<char> make_consts(const lbm_ctx *c)
{
    std::vector<char> raw(sizeof(CollideConsts<T>) * c->ninst);
    const lbm_params &p = c->p;
    const double s = (c->storage == LBM_F16S || c->storage == LBM_BF16S) ? p.storage_scale : 1.0;
    for (int k = 0; k < c->ninst; ++k) {
        CollideConsts<T> cc{};
        const double tau = c->itau[k];
        const double wp = 1.0 / tau;
        const double wm = p.collision == LBM_TRT ? 1.0 / (0.5 + p.magic / (tau - 0.5)) : wp;
        cc.rho0s = T(s * p.rho0);
        cc.ufac = T(1.0 / (s * p.rho0));
        const double *F = &c->iforce[size_t(3 * k)];
        for (int a = 0; a < 3; ++a) {
            cc.uoff[a] = T(F[a] / (2.0 * p.rho0));
            cc.Fs[a] = T(s * F[a]);
        }
        cc.omega_p = T(wp);
        cc.omega_m = T(wm);
        for (int q = 0; q < Q; ++q) {
            const double eu = ex(q) * p.wall_u[0] + ey(q) * p.wall_u[1] + ez(q) * p.wall_u[2];
            cc.bbw[q] = T(s * 6.0 * wq(q) * p.rho0 * eu);
        }
        cc.inv_s = T(1.0 / s);
        cc.rho0 = T(p.rho0);
        const double rho0s = s * p.rho0;
        const double ap = (1.0 - 0.5 * wp) / wp, am = (1.0 - 0.5 * wm) / wm;
        const double wc[2] = {1.0 / 18.0, 1.0 / 36.0};
        cc.zero = T(0);
        cc.nc15 = T(-1.5 * rho0s);
        cc.c45 = T(4.5 * rho0s);
        cc.c0a = T(wp / 3.0);
        cc.c0b = T(1.0 - wp);
        cc.hwp = T(0.5 * wp);
        cc.hwm = T(0.5 * wm);
        for (int a = 0; a < 3; ++a) {
            const double Fs = s * F[a];
            cc.Fs[a] = T(Fs);
            cc.k9F[a] = T(9.0 * ap * Fs);
            cc.nk3F[a] = T(-3.0 * ap * Fs);
        }
        for (int c2 = 0; c2 < 2; ++c2) {
            cc.obw[c2] = T(wp * wc[c2]);
            cc.oc3[c2] = T(wp * 3.0 * rho0s * wc[c2]);
            cc.nwpw[c2] = T(-wp * wc[c2]);
            cc.nwmc3[c2] = T(-wm * 3.0 * rho0s * wc[c2]);
            for (int a = 0; a < 3; ++a) {
                const double Fs = s * F[a];
                cc.okF[c2][a] = T(wp * 3.0 * am * wc[c2] * Fs);
                cc.nwmkF[c2][a] = T(-wm * 3.0 * am * wc[c2] * Fs);
            }
        }
        std::memcpy(raw.data() + sizeof(cc) * k, &cc, sizeof(cc));
    }
    return raw;
}

void invalidate_graphs(lbm_ctx *c)
{
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
}

// Tiles of the field and reduction kernels.
int set_tiles(lbm_ctx *c, const int t[3])
{
    std::vector<Tile> tiles;
    std::vector<long long> begin;
    build_tiles(c, t, tiles, begin);
    Tile *dt = nullptr;
    long long *db = nullptr;
    int rc = upload(c, &dt, tiles);
    if (rc) return rc;
    rc = upload(c, &db, begin);
    if (rc) return rc;
    size_t need = sizeof(double) * R_K * std::max<size_t>(tiles.size(), 1);
    if (need > c->partial_cap) {
        CK(cudaStreamSynchronize(c->stream), "set_tiles");
        disown(c, c->d_partial);
        c->d_partial = nullptr;
        c->partial_cap = 0;
        rc = own(c, &c->d_partial, need);
        if (rc) return rc;
        c->partial_cap = need;
    }
    CK(cudaStreamSynchronize(c->stream), "set_tiles");
    disown(c, c->d_tiles);
    disown(c, c->d_inst_begin);
    c->tiles.swap(tiles);
    c->inst_tile_begin.swap(begin);
    c->d_tiles = dt;
    c->d_inst_begin = db;
    for (int a = 0; a < 3; ++a) c->tile[a] = t[a];
    return LBM_OK;
}

// The sweep's work list: row tiles of t[0] x t[1] cells over t[2] z slices,
// or (flat > 0) runs of `flat` consecutive cells of each Block; grid > 0
// launches that many CTAs, which loop over the list.
int set_sweep(lbm_ctx *c, const int t[3], int flat, int grid, int pair)
{
    std::vector<Tile> st;
    std::vector<long long> unused;
    const int cpt = pair ? 2 : 1;  // cells per thread along x
    if (flat > 0) {
        for (size_t bi = 0; bi < c->blocks.size(); ++bi) {
            const BlockGeom &b = c->blocks[bi];
            const long long n = (long long)b.nx * b.ny * b.nz;
            for (long long i = 0; i < n; i += (long long)cpt * flat) st.push_back({int(bi), int(i), 0, 0});
        }
    } else {
        const int tc[3] = {cpt * t[0], t[1], t[2]};
        build_tiles(c, tc, st, unused);
    }
    // frozen instances (lbm_run_to_residual_each) are left out
    if (!c->active.empty()) {
        std::vector<Tile> kept;
        kept.reserve(st.size());
        for (const Tile &tl : st)
            if (c->active[size_t(c->blocks[size_t(tl.block)].inst)]) kept.push_back(tl);
        st.swap(kept);
    }
    Tile *dt = nullptr;
    int rc = upload(c, &dt, st);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream), "set_sweep");
    disown(c, c->d_stiles);
    c->d_stiles = dt;
    c->stiles.swap(st);
    c->flat = flat;
    c->grid = grid;
    c->pair = pair;
    if (flat > 0) {
        c->sw_tile[0] = flat;
        c->sw_tile[1] = c->sw_tile[2] = 1;
    } else {
        for (int a = 0; a < 3; ++a) c->sw_tile[a] = t[a];
    }
    invalidate_graphs(c);
    return LBM_OK;
}

// cuTensorMapEncodeTiled from the driver, fetched through the runtime (no
// link-time dependency on libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

int encode_map(lbm_ctx *c, CUtensorMap *m, CUtensorMapDataType dt, void *base, int esize, int pitch,
               long long plane, const BlockGeom &b, long long planes, int boxw, int boxh)
{
    auto enc = tensor_map_encoder();
    if (!enc) return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[4] = {cuuint64_t(pitch), cuuint64_t(b.py), cuuint64_t(b.nz + 2), cuuint64_t(planes)};
    cuuint64_t strides[3] = {cuuint64_t(pitch) * esize, cuuint64_t(pitch) * b.py * esize,
                             cuuint64_t(plane) * esize};
    cuuint32_t box[4] = {cuuint32_t(boxw), cuuint32_t(boxh), 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(m, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, LBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
    return LBM_OK;
}

// Whether the TMA sweep applies: one Patch of equal Blocks, 32/64/128 cells
// wide, a row count divisible by the strip height, FP32/F16S/BF16S.
bool tma_applicable(const lbm_ctx *c)
{
    if (c->ninst != 1 || c->storage == LBM_F64 || c->blocks.empty()) return false;
    const BlockGeom &b0 = c->blocks[0];
    if (b0.nx != 32 && b0.nx != 64 && b0.nx != 128) return false;
    if (b0.px != b0.nx) return false;
    if (b0.ny % (256 / b0.nx) != 0) return false;
    for (const BlockGeom &b : c->blocks)
        if (b.nx != b0.nx || b.ny != b0.ny || b.nz != b0.nz) return false;
    return true;
}

int setup_tma(lbm_ctx *c)
{
    const BlockGeom &b = c->blocks[0];
    const int tx = b.nx, ty = 256 / b.nx, A = 16 / c->elem;
    const CUtensorMapDataType dt = c->storage == LBM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : c->storage == LBM_F16S ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const long long planes = (long long)Q * (long long)c->blocks.size();
    // every Block has the same geometry, so Block k's plane q is plane 19k+q
    for (size_t k = 0; k < c->blocks.size(); ++k)
        if (c->blocks[k].pdf_base != (long long)k * Q * b.G)
            return fail(c, LBM_EINVAL, "TMA sweep: Blocks are not laid out uniformly");
    int rc;
    for (size_t k = 0; k < c->blocks.size(); ++k)
        if (c->blocks[k].cell_base != (long long)k * b.Gf)
            return fail(c, LBM_EINVAL, "TMA sweep: flag planes are not laid out uniformly");
    for (int par = 0; par < 2; ++par) {
        void *base = c->buf[par];
        if ((rc = encode_map(c, &c->maps.box_a[par], dt, base, c->elem, b.px, b.G, b, planes, tx, ty))) return rc;
        if ((rc = encode_map(c, &c->maps.box_b[par], dt, base, c->elem, b.px, b.G, b, planes, tx + A, ty)))
            return rc;
        if ((rc = encode_map(c, &c->maps.halo[par], dt, base, c->elem, b.px, b.G, b, planes, A, ty))) return rc;
    }
    if ((rc = encode_map(c, &c->maps.flags, CU_TENSOR_MAP_DATA_TYPE_UINT8, c->d_flags, 1, b.pxf, b.Gf, b,
                         (long long)c->blocks.size(), tx, ty)))
        return rc;
    int occ = 0, dev = 0, sms = 1;
    CK(tma_occupancy(c->storage, tx, c->p.collision, c->forced ? 1 : 0, &occ), "TMA occupancy");
    if (occ < 1) return fail(c, LBM_ECUDA, "TMA sweep does not fit on an SM");
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    c->tma_grid = occ * sms;
    c->kernel = LBM_KERNEL_TMA;
    return LBM_OK;
}

cudaError_t enqueue_aa_prepare(const lbm_ctx *c);

int build_context(lbm_ctx *c, const std::vector<InstSpec> &inst)
{
    const lbm_params &p = c->p;
    c->ninst = int(inst.size());
    c->storage = p.storage;
    c->elem = p.storage == LBM_F32 ? 4 : (p.storage == LBM_F64 ? 8 : 2);
    c->forced = p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0;
    for (int k = 0; k < c->ninst; ++k) c->iforce.insert(c->iforce.end(), p.force, p.force + 3);
    c->aa = p.streaming == LBM_STREAM_AA;
    c->sparse = p.layout == LBM_LAYOUT_SPARSE;
    if (c->sparse && (c->ninst != 1 || c->aa || p.kernel == LBM_KERNEL_TMA))
        return fail(c, LBM_EINVAL, "the fluid-cell list layout (LBM_LAYOUT_SPARSE) serves single Patches with "
                    "two-array streaming (not batches, LBM_STREAM_AA or LBM_KERNEL_TMA)");
    if (c->aa && (c->ninst != 1 || p.kernel == LBM_KERNEL_TMA))
        return fail(c, LBM_EINVAL, "in-place streaming (LBM_STREAM_AA) serves single Patches with the "
                    "register sweep (not batches, not LBM_KERNEL_TMA)");

    if (p.stream) {
        c->stream = static_cast<cudaStream_t>(p.stream);
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->own_stream = true;
    }

    // ---- blocks and flags
    std::vector<uint8_t> hflags;
    std::vector<uint32_t> hlinks;
    long long near_cells = 0;
    long long pdf_base = 0, cell_base = 0, out_base = 0;
    for (int k = 0; k < c->ninst; ++k) {
        const InstSpec &s = inst[k];
        c->idims.insert(c->idims.end(), s.dims, s.dims + 3);
        c->itau.push_back(s.tau);
        c->inst_out_base.push_back(out_base);
        const int nb[3] = {s.dims[0] / s.bdims[0], s.dims[1] / s.bdims[1], s.dims[2] / s.bdims[2]};
        const int first_block = int(c->blocks.size());
        for (int bz = 0; bz < nb[2]; ++bz)
            for (int by = 0; by < nb[1]; ++by)
                for (int bx = 0; bx < nb[0]; ++bx) {
                    BlockGeom b{};
                    b.xm_block = b.xp_block = -1;
                    b.nx = s.bdims[0];
                    b.ny = s.bdims[1];
                    b.nz = s.bdims[2];
                    b.px = round_up(b.nx, 32 / c->elem);
                    div_magic(uint32_t(b.nx), &b.mnx, &b.snx);
                    div_magic(uint32_t(b.ny), &b.mny, &b.sny);
                    b.xw_base[0] = b.xw_base[1] = -1;
                    b.pxf = round_up(OXF + b.nx + 1, 16);
                    b.py = b.ny + 2;
                    b.G = plane_cells((long long)b.px * b.py * (b.nz + 2), c->elem);
                    b.Gf = (long long)b.pxf * b.py * (b.nz + 2);
                    if ((long long)Q * b.G >= (1ll << 31))
                        return fail(c, LBM_EINVAL,
                                    "block of %dx%dx%d cells is too large for 32-bit plane "
                                    "offsets; split the domain into more blocks",
                                    b.nx, b.ny, b.nz);
                    b.pdf_base = pdf_base;
                    b.cell_base = cell_base;
                    b.inst = k;
                    b.gx = bx * b.nx;
                    b.gy = by * b.ny;
                    b.gz = bz * b.nz;
                    b.out_base = out_base;
                    b.NX = s.dims[0];
                    b.NY = s.dims[1];
                    b.NZ = s.dims[2];
                    pdf_base += (long long)Q * b.G;
                    cell_base += b.Gf;
                    // flags of every stored cell (interior, ghost shell, padding)
                    std::vector<uint8_t> f(size_t(b.Gf), F_NOSLIP);
                    for (int z = -1; z <= b.nz; ++z)
                        for (int y = -1; y <= b.ny; ++y)
                            for (int x = -1; x <= b.nx; ++x) {
                                const long long cidx =
                                    ((long long)(z + 1) * b.py + (y + 1)) * b.pxf + (x + OXF);
                                uint8_t v = classify(p, s.dims, s.flags, b.gx + x, b.gy + y, b.gz + z);
                                if (v > F_PRESSURE)
                                    return fail(c, LBM_EINVAL,
                                                "flag value %d is not LBM_FLUID/NOSLIP/MOVING/PRESSURE", int(v));
                                if (v == F_PRESSURE) c->has_pressure = true;
                                f[cidx] = v;
                            }
                    const long long pxy = (long long)b.pxf * b.py;
                    std::vector<uint32_t> lk(size_t(b.Gf), 0u);
                    for (int z = 0; z < b.nz; ++z)
                        for (int y = 0; y < b.ny; ++y)
                            for (int x = 0; x < b.nx; ++x) {
                                const long long cidx = (z + 1) * pxy + (long long)(y + 1) * b.pxf + (x + OXF);
                                if (f[cidx] != F_FLUID) continue;
                                ++c->fluid;
                                uint32_t m = 0;
                                for (int q = 1; q < Q; ++q) {
                                    const uint8_t nk =
                                        f[cidx - (ex(q) + ey(q) * (long long)b.pxf + ez(q) * pxy)] & F_KIND;
                                    if (nk) m |= 1u << q;
                                    if (nk == F_MOVING) m |= L_MOVING;
                                    if (nk == F_PRESSURE) m |= L_PRESSURE;
                                }
                                if (m) {
                                    f[cidx] |= F_NEAR;
                                    lk[cidx] = m;
                                    ++near_cells;
                                }
                            }
                    // FP32 and 16-bit: no-slip cells that share a 32-byte PDF sector
                    // with a fluid cell store the rest state in the one-cell sweep, and
                    // (FP32) the last cells of a row zero its padding, so that every
                    // sector the sweep writes is complete (a partly written sector
                    // costs the memory system a read of the old sector; the 16-bit
                    // sweeps ran slower with padding stores in their kernels)
                    if (c->storage != LBM_F64)
                        mark_sector_fills(f.data(), b.nx, b.ny, b.nz, b.px, b.py, b.pxf, c->elem,
                                          c->storage == LBM_F32);
                    hflags.insert(hflags.end(), f.begin(), f.end());
                    hlinks.insert(hlinks.end(), lk.begin(), lk.end());
                    c->blocks.push_back(b);
                }
        // ---- direct reads across x faces
        for (int bz = 0; bz < nb[2]; ++bz)
            for (int by = 0; by < nb[1]; ++by)
                for (int bx = 0; bx < nb[0]; ++bx) {
                    BlockGeom &b = c->blocks[first_block + (bz * nb[1] + by) * nb[0] + bx];
                    for (int side = -1; side <= 1; side += 2) {
                        int nbx = bx + side;
                        if (nbx < 0 || nbx >= nb[0]) {
                            if (!p.periodic[0]) continue;
                            nbx = (nbx + nb[0]) % nb[0];
                        }
                        const int nid = first_block + (bz * nb[1] + by) * nb[0] + nbx;
                        const BlockGeom &n = c->blocks[nid];
                        const long long off = n.pdf_base - b.pdf_base - side * (long long)b.nx;
                        if (side < 0) {
                            b.xm_off = off;
                            b.xm_block = nid;
                        } else {
                            b.xp_off = off;
                            b.xp_block = nid;
                        }
                    }
                }
        // ---- in place: side storage beyond wall x faces
        if (c->aa)
            for (int bi = first_block; bi < int(c->blocks.size()); ++bi) {
                BlockGeom &b = c->blocks[bi];
                const long long rows = (long long)b.py * (b.nz + 2);
                for (int side = 0; side < 2; ++side)
                    if ((side == 0 ? b.xm_block : b.xp_block) < 0) {
                        b.xw_base[side] = pdf_base;
                        pdf_base += 5 * rows;
                    }
            }
        // ---- ghost exchange plan: faces and edges with a neighbour block
        for (int bz = 0; bz < nb[2]; ++bz)
            for (int by = 0; by < nb[1]; ++by)
                for (int bx = 0; bx < nb[0]; ++bx) {
                    const int me = first_block + (bz * nb[1] + by) * nb[0] + bx;
                    const int bpos[3] = {bx, by, bz};
                    for (int n0 = -1; n0 <= 1; ++n0)
                        for (int n1 = -1; n1 <= 1; ++n1)
                            for (int n2 = -1; n2 <= 1; ++n2) {
                                const int n[3] = {n0, n1, n2};
                                const int nnz = (n0 != 0) + (n1 != 0) + (n2 != 0);
                                if (nnz == 0 || nnz == 3) continue;  // no corner links in D3Q19
                                if (n0 != 0) continue;  // x faces: read directly by the sweep
                                int npos[3];
                                bool ok = true;
                                for (int a = 0; a < 3; ++a) {
                                    npos[a] = bpos[a] + n[a];
                                    if (npos[a] < 0 || npos[a] >= nb[a]) {
                                        if (!p.periodic[a]) ok = false;
                                        npos[a] = (npos[a] + nb[a]) % nb[a];
                                    }
                                }
                                if (!ok) continue;
                                // one slab per direction entering this Block
                                // through the face / edge: the ghost rows of
                                // `me`, copied from the neighbour's boundary rows
                                const BlockGeom &bm = c->blocks[me];
                                const BlockGeom &bs =
                                    c->blocks[first_block + (npos[2] * nb[1] + npos[1]) * nb[0] + npos[0]];
                                const int yg = n1 < 0 ? -1 : (n1 > 0 ? bm.ny : 0);
                                const int zg = n2 < 0 ? -1 : (n2 > 0 ? bm.nz : 0);
                                const int ys = yg - n1 * bm.ny, zs = zg - n2 * bm.nz;
                                const long long pxy = (long long)bm.px * bm.py;
                                XSlab sl{};
                                sl.len = bm.px;  // whole rows (padding included) stay 32-byte aligned
                                if (n1 != 0 && n2 == 0) {  // y face: one row per z
                                    sl.rows = bm.nz;
                                    sl.stride = pxy;
                                } else if (n2 != 0 && n1 == 0) {  // z face: one row per y
                                    sl.rows = bm.ny;
                                    sl.stride = bm.px;
                                } else {  // yz edge
                                    sl.rows = 1;
                                    sl.stride = 0;
                                }
                                const long long d0 = ((long long)(zg + 1) * bm.py + (yg + 1)) * bm.px;
                                const long long s0 = ((long long)(zs + 1) * bm.py + (ys + 1)) * bm.px;
                                for (int q = 1; q < Q; ++q) {
                                    const int e[3] = {ex(q), ey(q), ez(q)};
                                    bool into = true, out = true;
                                    for (int a2 = 0; a2 < 3; ++a2) {
                                        if (n[a2] != 0 && e[a2] != -n[a2]) into = false;
                                        if (n[a2] != 0 && e[a2] != n[a2]) out = false;
                                    }
                                    if (c->aa) {
                                        // in place: the odd step reads and writes the directions
                                        // leaving this Block through the face / edge
                                        if (!out) continue;
                                        // forward: into fluid ghost cells only (a wall or
                                        // pressure node's slots hold what this Block's
                                        // own cells stored there)
                                        XSlabF fw{};
                                        fw.len = bm.nx;
                                        fw.rows = sl.rows;
                                        fw.stride = sl.stride;
                                        fw.dst = bm.pdf_base + (long long)q * bm.G + d0;
                                        fw.src = bs.pdf_base + (long long)q * bs.G + s0;
                                        fw.fstride = n1 != 0 && n2 == 0 ? (long long)bm.pxf * bm.py
                                                     : (n2 != 0 && n1 == 0 ? bm.pxf : 0);
                                        fw.fsrc = bm.cell_base +
                                                  ((long long)(zg + 1) * bm.py + (yg + 1)) * bm.pxf + OXF;
                                        c->aa_fwd.push_back(fw);
                                        // reverse: only rows whose streaming cell (ghost - e_q)
                                        // lies inside this Block along the slab's row axis
                                        XSlabF rv{};
                                        rv.len = bm.nx;
                                        long long r0 = 0;  // first row
                                        if (n1 != 0 && n2 == 0) {
                                            r0 = std::max(0, e[2]);
                                            rv.rows = bm.nz - std::abs(e[2]);
                                            rv.stride = pxy;
                                            rv.fstride = (long long)bm.pxf * bm.py;
                                        } else if (n2 != 0 && n1 == 0) {
                                            r0 = std::max(0, e[1]);
                                            rv.rows = bm.ny - std::abs(e[1]);
                                            rv.stride = bm.px;
                                            rv.fstride = bm.pxf;
                                        } else {
                                            rv.rows = 1;
                                        }
                                        const long long roff = r0 * rv.stride;
                                        rv.src = bm.pdf_base + (long long)q * bm.G + d0 + roff;
                                        rv.dst = bs.pdf_base + (long long)q * bs.G + s0 + roff;
                                        // flag of the streaming cell of element (row 0, x = 0)
                                        const long long yw = (n1 != 0 ? yg : r0 * (n2 != 0)) - e[1];
                                        const long long zw = (n2 != 0 ? zg : r0 * (n1 != 0)) - e[2];
                                        rv.fsrc = bm.cell_base + ((zw + 1) * bm.py + (yw + 1)) * bm.pxf + OXF - e[0];
                                        if (rv.rows > 0) c->aa_rev.push_back(rv);
                                        c->exchange_pdfs += 2ll * sl.rows * bm.nx;
                                        continue;
                                    }
                                    if (!into) continue;
                                    sl.dst = bm.pdf_base + (long long)q * bm.G + d0;
                                    sl.src = bs.pdf_base + (long long)q * bs.G + s0;
                                    c->xslabs.push_back(sl);
                                    c->exchange_pdfs += (long long)sl.rows * bm.nx;
                                }
                            }
                }
        out_base += (long long)s.dims[0] * s.dims[1] * s.dims[2];
    }
    c->cells = out_base;
    c->stored = cell_base;

    // ---- fluid-cell list layout: numbering, neighbour table (periodic images
    // and Block faces resolved here, so no exchange runs)
    std::vector<int> hsidx, hnbr;
    if (c->sparse) {
        c->xslabs.clear();
        c->exchange_pdfs = 0;
        hsidx.assign(size_t(cell_base), -1);
        long long nf = 0;
        for (const BlockGeom &b : c->blocks)
            for (int z = 0; z < b.nz; ++z)
                for (int y = 0; y < b.ny; ++y)
                    for (int x = 0; x < b.nx; ++x) {
                        const long long cf = ((long long)(z + 1) * b.py + (y + 1)) * b.pxf + x + OXF;
                        const size_t at = size_t(b.cell_base + cf);
                        if ((hflags[at] & F_KIND) == F_FLUID) hsidx[at] = int(nf++);
                    }
        const long long stride = std::max<long long>(64, (nf + 63) / 64 * 64);
        if ((long long)Q * stride >= (1ll << 31))
            return fail(c, LBM_EINVAL, "fluid-cell list of %lld cells: 19 x cells must stay below 2^31", nf);
        c->nfluid = nf;
        c->nstride = stride;
        hnbr.assign(size_t(Q * stride), -1);
        const InstSpec &s0 = inst[0];
        const int *N = s0.dims;
        const int nb[3] = {N[0] / s0.bdims[0], N[1] / s0.bdims[1], N[2] / s0.bdims[2]};
        for (const BlockGeom &b : c->blocks)
            for (int z = 0; z < b.nz; ++z)
                for (int y = 0; y < b.ny; ++y)
                    for (int x = 0; x < b.nx; ++x) {
                        const long long cf = ((long long)(z + 1) * b.py + (y + 1)) * b.pxf + x + OXF;
                        const int k = hsidx[size_t(b.cell_base + cf)];
                        if (k < 0) continue;
                        int pres = 0;
                        for (int q = 1; q < Q; ++q) {
                            long long P[3] = {b.gx + x - ex(q), b.gy + y - ey(q), b.gz + z - ez(q)};
                            const int kind = classify(p, N, s0.flags, P[0], P[1], P[2]) & F_KIND;
                            int code = kind == F_MOVING ? -2 : (kind == F_PRESSURE ? -3 : -1);
                            if (kind == F_PRESSURE) pres = 1;
                            if (kind == F_FLUID) {
                                for (int a2 = 0; a2 < 3; ++a2) P[a2] = ((P[a2] % N[a2]) + N[a2]) % N[a2];
                                const int bd[3] = {s0.bdims[0], s0.bdims[1], s0.bdims[2]};
                                const BlockGeom &n = c->blocks[size_t(((P[2] / bd[2]) * nb[1] + P[1] / bd[1]) * nb[0] +
                                                                      P[0] / bd[0])];
                                const long long ncf = ((P[2] % bd[2] + 1) * n.py + (P[1] % bd[1] + 1)) * n.pxf +
                                                      P[0] % bd[0] + OXF;
                                code = hsidx[size_t(n.cell_base + ncf)];
                            }
                            hnbr[size_t(q * stride + k)] = code;
                        }
                        hnbr[size_t(k)] = pres;
                    }
    }

    // ---- device memory
    const size_t buf_bytes = (c->sparse ? size_t(Q * c->nstride) : size_t(pdf_base)) * c->elem;
    c->buf_bytes = buf_bytes;
    int rc;
    if ((rc = own(c, &c->buf[0], buf_bytes))) return rc;
    CK(cudaMemsetAsync(c->buf[0], 0, buf_bytes, c->stream), "memset");
    if (!c->aa) {  // in place: one array
        if ((rc = own(c, &c->buf[1], buf_bytes))) return rc;
        CK(cudaMemsetAsync(c->buf[1], 0, buf_bytes, c->stream), "memset");
    }
    if ((rc = upload(c, &c->d_flags, hflags))) return rc;
    if ((rc = upload(c, &c->d_links, hlinks))) return rc;
    if ((rc = upload(c, &c->d_blocks, c->blocks))) return rc;
    if ((rc = upload(c, &c->d_xslabs, c->xslabs))) return rc;
    if ((rc = upload(c, &c->d_aa_fwd, c->aa_fwd))) return rc;
    if ((rc = upload(c, &c->d_aa_rev, c->aa_rev))) return rc;
    if (c->sparse) {
        if ((rc = upload(c, &c->d_sidx, hsidx))) return rc;
        if ((rc = upload(c, &c->d_nbr, hnbr))) return rc;
    }
    std::vector<char> consts =
        c->storage == LBM_F64 ? make_consts<double>(c) : make_consts<float>(c);
    c->h_consts = consts;
    if ((rc = upload(c, reinterpret_cast<char **>(&c->d_consts), consts))) return rc;
    if ((rc = own(c, &c->d_red, sizeof(double) * R_K * c->ninst))) return rc;
    if ((rc = own(c, &c->d_err, sizeof(int)))) return rc;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "memset");

    // default tile: a warp multiple along x covering the block width, 256 threads
    int maxnx = 0;
    for (const BlockGeom &b : c->blocks) maxnx = std::max(maxnx, b.nx);
    int td[3];
    td[0] = std::min(128, round_up(std::max(maxnx, 1), 32));
    td[1] = std::max(1, 256 / td[0]);
    td[2] = 4;
    if ((rc = set_tiles(c, td))) return rc;
    int t[3] = {p.tile[0], p.tile[1], p.tile[2]};
    int flat = 0, pair = 0;
    bool budget5 = false;
    if (t[0] <= 0 || t[1] <= 0 || t[2] <= 0) {
        for (int a = 0; a < 3; ++a) t[a] = td[a];
        // Two cells per thread wherever the Block widths are even (FP32 and
        // 16-bit storage): twice the bytes in flight per thread.  Blocks whose
        // width is not a multiple of the tile's cells would leave lanes of
        // every row tile idle: sweep them in runs of consecutive cells.  Porous
        // media (more than 10% near-wall cells) put near-wall cells in most
        // pairs, whose per-cell pulls make the pair slower than one cell per
        // thread (measured on 48 sphere-packed 64^3 channels: 0.65 against
        // 0.43 ms per sweep in FP32, 0.49 against 0.37 ms in F16S).
        bool even = c->storage != LBM_F64, w64 = true, w32 = true;
        for (const BlockGeom &b : c->blocks) {
            even = even && (b.nx % 2 == 0);
            w64 = w64 && (b.nx % 64 == 0);
            w32 = w32 && (b.nx % 32 == 0);
        }
        const bool porous = near_cells * 10 > c->fluid;
        if (c->aa) {  // in place: one cell per thread (two spill at these register budgets)
            if (!w32) flat = 256;
        } else if (porous) {
            flat = 128;
            // FP32 PDFs leave the one-cell sweep room for a 48-register budget
            // (five 256-thread CTAs per SM): measured 0.415 against 0.439 ms per
            // sweep on 48 sphere-packed 64^3 channels, 1.65 against 1.69 ms on
            // 256 of them; 16-bit storage needs its conversion registers and
            // stays at budget 4 (0.445 against 0.363 ms)
            budget5 = c->storage == LBM_F32 && !c->sparse;
        } else if (even && w64) {
            pair = 1;
            t[0] = 32;
            t[1] = 4;
            t[2] = 2;
        } else if (even) {
            pair = 1;
            flat = 128;
        } else if (!w32) {
            flat = 256;
        }
    }
    if (t[0] * t[1] > 256 || t[0] % 32 != 0)
        return fail(c, LBM_EINVAL, "tile %dx%d: threads along x must be a multiple of 32 and "
                    "tile[0]*tile[1] <= 256", t[0], t[1]);
    if ((rc = set_sweep(c, t, flat, 0, pair))) return rc;
    // link masks pay where near-wall and interior cells share warps
    c->mask = !c->aa && near_cells * 10 > c->fluid ? 1 : 0;
    // the TMA sweep is set up wherever it applies (lbm_autotune may pick it);
    // it runs by default only when requested: the register sweep is faster
    // on GB300 for every workload measured so far
    if (p.kernel != LBM_KERNEL_REGISTER && !c->aa && tma_applicable(c)) {
        if ((rc = setup_tma(c))) return rc;
        if (p.kernel == LBM_KERNEL_AUTO) c->kernel = LBM_KERNEL_REGISTER;
    } else if (p.kernel == LBM_KERNEL_TMA) {
        return fail(c, LBM_EINVAL, "the TMA sweep needs one Patch of equal Blocks 32, 64 or 128 "
                    "cells wide with rows divisible by 256/width, and F32/F16S/BF16S storage");
    }

    if (budget5 && c->kernel == LBM_KERNEL_REGISTER) c->minb = 5;

    // in place: the rest state's pressure links
    CK(enqueue_aa_prepare(c), "prepare pressure links");

    // graph length: enough work per replay to hide launch overhead
    if (p.graph_steps < 0) {
        c->graph_steps = 0;
    } else if (p.graph_steps > 0) {
        c->graph_steps = p.graph_steps + (p.graph_steps & 1);
    } else {
        long long per = std::max<long long>(c->cells, 1);
        long long g = (4ll << 20) / per;
        g = std::max(2ll, std::min(100ll, g + (g & 1)));
        c->graph_steps = int(g);
    }
    CK(cudaStreamSynchronize(c->stream), "create");
    return LBM_OK;
}

template std::vector<char> make_consts<float>(const lbm_ctx *c);
template std::vector<char> make_consts<double>(const lbm_ctx *c);

}  // namespace rt
}  // namespace lbm
