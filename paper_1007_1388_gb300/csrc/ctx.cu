// Host runtime of liblbm.so: contexts, the Patch/Block manager, the ghost
// exchange plan, CUDA-graph replay of time steps, launch timing, the tile
// autotuner and the C ABI of include/lbm.h.
//
// A context holds one Patch split into Blocks (Sec. 4.2), or a batch of
// independent single-Block instances.  All Blocks of all instances live in
// two device buffers (src / dst, Sec. 2.1 two-grid pull scheme), each Block
// with a one-cell ghost shell.  One time step is one Sweep (Sec. 4): the
// communication step (exchange kernel, device memory only; the local
// "buffer swap" of Sec. 4.4 becomes a direct ghost-layer copy) followed by the
// work step (sweep kernel over every Block in one launch).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <memory>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include <cudaTypedefs.h>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

// ------------------------------------------------------------ allocator
struct Allocator {
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void *user = nullptr;
};
Allocator g_alloc;
thread_local std::string g_create_error;
std::mutex g_alloc_mu;

struct DevMem {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

namespace lbm {
void *tma_encode_fn()
{
    static void *fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = p;
        else
            cudaGetLastError();
    }
    return fn;
}

void current_allocator(lbm_alloc_fn *alloc, lbm_free_fn *release, void **user)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    *alloc = g_alloc.alloc;
    *release = g_alloc.release;
    *user = g_alloc.user;
}
}  // namespace lbm

struct lbm_ctx {
    // configuration
    lbm_params p{};
    int ninst = 0;
    std::vector<int> idims;        // 3 per instance
    std::vector<double> itau;
    std::vector<double> iforce;    // 3 per instance (lbm_params.force, or lbm_set_forces)
    int storage = LBM_F32;
    int elem = 4;
    bool forced = false;
    // geometry (host copies)
    std::vector<BlockGeom> blocks;
    std::vector<Tile> tiles;
    std::vector<long long> inst_tile_begin;
    std::vector<XSlab> xslabs;
    std::vector<long long> inst_out_base;
    long long cells = 0, fluid = 0, stored = 0, exchange_pdfs = 0;
    int tile[3] = {64, 4, 4};     // tiles of the field and reduction kernels (fixed at create)
    // the sweep's own work list (lbm_autotune changes only this)
    int sw_tile[3] = {64, 4, 4};  // row tile, or {flat, 1, 1}
    int flat = 0;                 // > 0: runs of this many consecutive cells per CTA
    int grid = 0;                 // 0 = one CTA per tile, else a persistent grid
    int mask = 0;                 // near-wall cells via link masks under a warp vote
    int pair = 0;                 // two neighbouring cells per thread (FP32 / 16-bit storage)
    std::vector<Tile> stiles;
    std::vector<char> active;     // per instance: swept (1) or frozen (0)
    int minb = 4;  // register budget of the sweep (resident CTAs per SM)
    std::vector<char> h_consts;  // host copy of the per-instance CollideConsts
    bool has_pressure = false;   // some cell or wall of the Patch is a pressure boundary
    // curved walls (lbm_set_wall_distances): link table and per-flag-cell rows
    bool has_curved = false;
    long long curved_links = 0;
    int *d_curv_idx = nullptr;
    void *d_curv_q = nullptr;
    // in-place streaming (LBM_STREAM_AA): one PDF array; aa_phase 0 when it
    // holds the state swapped in the cells' own slots (read through a slot
    // remap), 1 after an odd number of steps, when it holds the state
    // streamed (read back into a temporary array)
    bool aa = false;
    int aa_phase = 0;
    size_t buf_bytes = 0;         // bytes of one PDF array
    std::vector<XSlabF> aa_fwd;   // ghost rows <- neighbours' boundary rows, before the odd step
    std::vector<XSlabF> aa_rev;   // neighbours' boundary rows <- ghost rows, after it
    XSlabF *d_aa_fwd = nullptr;
    XSlabF *d_aa_rev = nullptr;
    // fluid-cell list layout (LBM_LAYOUT_SPARSE): list index per flag cell,
    // neighbour table [19][nstride]
    bool sparse = false;
    long long nfluid = 0, nstride = 0;
    int *d_sidx = nullptr;
    int *d_nbr = nullptr;
    // kernel choice and the TMA sweep's launch state
    int kernel = LBM_KERNEL_REGISTER;
    TmaMaps maps{};
    int tma_zchunk = 8;
    int tma_grid = 0;
    int *d_err = nullptr;       // device error word written by timed-out waits
    // device
    Allocator alloc;
    std::vector<DevMem> owned;
    void *buf[2] = {nullptr, nullptr};
    uint8_t *d_flags = nullptr;
    uint32_t *d_links = nullptr;
    BlockGeom *d_blocks = nullptr;
    Tile *d_tiles = nullptr;
    Tile *d_stiles = nullptr;
    XSlab *d_xslabs = nullptr;
    void *d_consts = nullptr;
    long long *d_inst_begin = nullptr;
    double *d_partial = nullptr;
    float *d_snap = nullptr;       // velocity snapshot: rho [cells] then u [3 cells]
    double *d_red = nullptr;
    size_t partial_cap = 0;
    long long device_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // state
    int cur = 0;
    bool have_prev = false;
    // graphs: graph[par] runs graph_steps steps starting from buffer par
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps = 0;
    // launch timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev;   // 3 per profiled step
    std::vector<char> ev_has_x;
    size_t ev_used = 0;
    double acc_sweep_ms = 0, acc_x_ms = 0;
    long long acc_sweeps = 0, acc_x = 0;
    std::string err;
};

namespace {

int fail(lbm_ctx *c, int code, const char *fmt, ...)
{
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    if (c)
        c->err = msg;
    else
        g_create_error = msg;
    return code;
}

int cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

void *dev_alloc(lbm_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->alloc.alloc) {
        p = c->alloc.alloc(bytes, (void *)c->stream, c->alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(lbm_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    if (c->alloc.release)
        c->alloc.release(p, bytes, (void *)c->stream, c->alloc.user);
    else if (!c->alloc.alloc)
        cudaFree(p);
}

// Allocation owned by the context until lbm_destroy.
template <typename P>
int own(lbm_ctx *c, P **out, size_t bytes)
{
    void *p = dev_alloc(c, bytes);
    if (!p) return fail(c, LBM_ENOMEM, "device allocation of %zu bytes failed", bytes);
    c->owned.push_back({p, bytes});
    c->device_bytes += (long long)bytes;
    *out = static_cast<P *>(p);
    return LBM_OK;
}

// Releases one allocation made with own() (no-op for NULL).
void disown(lbm_ctx *c, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < c->owned.size(); ++i)
        if (c->owned[i].ptr == p) {
            dev_free(c, p, c->owned[i].bytes);
            c->device_bytes -= (long long)c->owned[i].bytes;
            c->owned.erase(c->owned.begin() + long(i));
            return;
        }
}

// Scoped temporary device buffer.
struct Temp {
    lbm_ctx *c;
    void *p = nullptr;
    size_t bytes = 0;
    Temp(lbm_ctx *c_, size_t b) : c(c_), bytes(b) { p = dev_alloc(c, b); }
    ~Temp() { dev_free(c, p, bytes); }
};

template <typename T>
int upload(lbm_ctx *c, T **dst, const std::vector<T> &v)
{
    int rc = own(c, dst, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (rc) return rc;
    if (!v.empty())
        CK(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c->stream),
           "upload");
    return LBM_OK;
}

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

// Instance description used while building a context.
struct InstSpec {
    int dims[3];
    int bdims[3];
    double tau;
    const uint8_t *flags;
};

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
int set_sweep(lbm_ctx *c, const int t[3], int flat, int grid, int pair = 0)
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
    if (t[0] <= 0 || t[1] <= 0 || t[2] <= 0) {
        for (int a = 0; a < 3; ++a) t[a] = td[a];
        // Two cells per thread wherever the Block widths are even (FP32 and
        // 16-bit storage): twice the bytes in flight per thread.  Blocks whose
        // width is not a multiple of the tile's cells would leave lanes of
        // every row tile idle: sweep them in runs of consecutive cells.
        bool even = c->storage != LBM_F64, w64 = true, w32 = true;
        for (const BlockGeom &b : c->blocks) {
            even = even && (b.nx % 2 == 0);
            w64 = w64 && (b.nx % 64 == 0);
            w32 = w32 && (b.nx % 32 == 0);
        }
        if (c->aa) {  // in place: one cell per thread (two spill at these register budgets)
            if (!w32) flat = 256;
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

// ---- launches
SweepArgs sweep_args(const lbm_ctx *c, int from)
{
    SweepArgs a{};
    a.tiles = c->d_stiles;
    a.ntiles = (long long)c->stiles.size();
    a.blocks = c->d_blocks;
    a.consts = c->d_consts;
    a.flags = c->d_flags;
    a.links = c->d_links;
    a.src = c->buf[from];
    a.dst = c->buf[from ^ 1];
    a.tx = c->sw_tile[0];
    a.ty = c->sw_tile[1];
    a.tz = c->sw_tile[2];
    a.flat = c->flat > 0 ? 1 : 0;
    a.mask = c->mask;
    a.pair = c->pair;
    a.collision = c->p.collision;
    a.forced = c->forced ? 1 : 0;
    a.storage = c->storage;
    a.grid = c->grid;
    a.minb = c->minb;
    a.unif = c->ninst == 1 ? 1 : 0;
    {
        const double sc = (c->storage == LBM_F16S || c->storage == LBM_BF16S) ? c->p.storage_scale : 1.0;
        const double rho_b = c->p.rho_b > 0.0 ? c->p.rho_b : c->p.rho0;
        a.pbd = 2.0 * sc * (rho_b - c->p.rho0);
        a.pbf = float(a.pbd);
        a.pres = (c->has_pressure ? 1 : 0) | (c->has_curved ? 2 : 0);
        a.curv_idx = c->d_curv_idx;
        a.curv_q = c->d_curv_q;
        a.nbr = c->d_nbr;
        a.nfluid = c->nfluid;
        a.nstride = c->nstride;
    }
    if (a.unif) {
        if (c->storage == LBM_F64)
            std::memcpy(&a.kd, c->h_consts.data(), sizeof(a.kd));
        else
            std::memcpy(&a.kf, c->h_consts.data(), sizeof(a.kf));
    }
    return a;
}

FieldArgs field_args(const lbm_ctx *c)
{
    FieldArgs a{};
    a.tiles = c->d_tiles;
    a.ntiles = (long long)c->tiles.size();
    a.blocks = c->d_blocks;
    a.consts = c->d_consts;
    a.flags = c->d_flags;
    a.tx = c->tile[0];
    a.ty = c->tile[1];
    a.tz = c->tile[2];
    a.storage = c->storage;
    a.sidx = c->sparse ? c->d_sidx : nullptr;
    a.sstride = c->nstride;
    return a;
}

// Field arguments for a call that writes the state where it is: in place, an
// even-time array (slots swapped).
FieldArgs write_args(const lbm_ctx *c)
{
    FieldArgs a = field_args(c);
    a.swap = c->aa ? 1 : 0;
    return a;
}

cudaError_t enqueue_exchange(const lbm_ctx *c, int which)
{
    ExchangeArgs x{};
    x.slabs = c->d_xslabs;
    x.nslabs = int(c->xslabs.size());
    x.buf = c->buf[which];
    x.elem_bytes = c->elem;
    return launch_exchange(x, c->stream);
}

// Bound of every mbarrier wait of the TMA sweep, in SM clock cycles (about
// one second at the GB300's 2 GHz boost clock).
constexpr long long kWaitCycles = 2000000000ll;

// The work step from buffer `from` into the other.
cudaError_t enqueue_sweep(const lbm_ctx *c, int from)
{
    SweepArgs a = sweep_args(c, from);
    if (c->sparse) return launch_sweep_sparse(a, c->stream);
    if (c->kernel != LBM_KERNEL_TMA) return launch_sweep(a, c->stream);
    const BlockGeom &b = c->blocks[0];
    TmaSweepArgs t{};
    t.a = a;
    t.nx = b.nx;
    t.ny = b.ny;
    t.nz = b.nz;
    t.px = b.px;
    t.py = b.py;
    t.pxf = b.pxf;
    t.ngy = b.ny / (256 / b.nx);
    t.zchunk = c->tma_zchunk;
    t.nzc = (b.nz + c->tma_zchunk - 1) / c->tma_zchunk;
    t.nitems = (long long)c->blocks.size() * t.ngy * t.nzc;
    t.parity = from;
    t.drop_stage = (c->p.debug_flags & LBM_DEBUG_DROP_STAGE) ? 3 : -1;
    t.wait_cycles = kWaitCycles;
    t.err = c->d_err;
    const int grid = int(std::min<long long>(t.nitems, c->tma_grid));
    return launch_sweep_tma(t, c->maps, grid, c->stream);
}

bool exchange_each_step(const lbm_ctx *c)
{
    return !c->xslabs.empty();
}

// In-place scheme: the forward exchange (before an odd step, and before a
// gather), the reverse exchange (after an odd step), and the sweep itself.
cudaError_t enqueue_aa_fwd(const lbm_ctx *c)
{
    return launch_exchange_flagged(c->d_aa_fwd, int(c->aa_fwd.size()), c->buf[0], c->elem, c->d_flags,
                                   c->stream);
}

cudaError_t enqueue_aa_rev(const lbm_ctx *c)
{
    return launch_exchange_flagged(c->d_aa_rev, int(c->aa_rev.size()), c->buf[0], c->elem, c->d_flags,
                                   c->stream);
}

cudaError_t enqueue_aa_sweep(const lbm_ctx *c, int mode, void *gather_dst = nullptr)
{
    SweepArgs a = sweep_args(c, 0);
    a.src = c->buf[0];
    a.dst = mode == 2 ? gather_dst : c->buf[0];
    return launch_sweep_aa(a, mode, c->stream);
}

// One in-place step from phase ph: from an even time the forward exchange,
// the pull-and-push step and the reverse exchange; from an odd time the
// local step.
cudaError_t enqueue_aa_step(const lbm_ctx *c, int ph)
{
    if (ph == 1) return enqueue_aa_sweep(c, 0);
    cudaError_t e = enqueue_aa_fwd(c);
    if (e == cudaSuccess) e = enqueue_aa_sweep(c, 1);
    if (e == cudaSuccess) e = enqueue_aa_rev(c);
    return e;
}

// One step from buffer `from` (communication step, then the work step); in
// place, `from` is the phase.
cudaError_t enqueue_step(const lbm_ctx *c, int from)
{
    if (c->aa) return enqueue_aa_step(c, from);
    if (exchange_each_step(c)) {
        cudaError_t e = enqueue_exchange(c, from);
        if (e != cudaSuccess) return e;
    }
    return enqueue_sweep(c, from);
}

// Reads and clears the device error word (synchronises the stream).
int check_device_error(lbm_ctx *c)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error word");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (h == 0) return LBM_OK;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream), "memset");
    CK(cudaStreamSynchronize(c->stream), "sync");
    return fail(c, LBM_ETIMEOUT, "a bounded wait of the TMA sweep expired (%s); the state is undefined",
                h == 1 ? "staged data never arrived" : h == 2 ? "a stage was never released"
                                                                : "copies in flight at exit");
}

// In place, after the state was written at an even time: the values that
// the next step pulls over pressure links (stored in the pressure nodes'
// slots; the steps themselves keep them current).
cudaError_t enqueue_aa_prepare(const lbm_ctx *c)
{
    if (!c->aa || !c->has_pressure) return cudaSuccess;
    return enqueue_aa_sweep(c, 4);
}

// The odd-time state of the in-place scheme read back into the natural
// layout of `dst` (S_q(x) at slot q).
cudaError_t enqueue_aa_gather(const lbm_ctx *c, void *dst)
{
    cudaError_t e = cudaMemsetAsync(dst, 0, c->buf_bytes, c->stream);
    if (e == cudaSuccess) e = enqueue_aa_sweep(c, 2, dst);
    return e;
}

// The state for reading: the PDF array itself (with `fa.swap` set at an even
// time of the in-place scheme), or, at an odd time, a copy in the natural
// layout owned by `t`.
int readable_state(lbm_ctx *c, std::unique_ptr<Temp> &t, const void **state, FieldArgs &fa)
{
    fa.swap = 0;
    if (!c->aa || c->aa_phase == 0) {
        *state = c->buf[c->cur];
        fa.swap = c->aa ? 1 : 0;
        return LBM_OK;
    }
    t.reset(new Temp(c, c->buf_bytes));
    if (!t->p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes (the in-place state read back)", t->bytes);
    CK(enqueue_aa_gather(c, t->p), "gather launch");
    *state = t->p;
    return LBM_OK;
}

// Brings the in-place array to an even-time layout (before a call that
// changes the state where it is): read back, then stored swapped.
int aa_normalize(lbm_ctx *c)
{
    if (!c->aa || c->aa_phase == 0) return LBM_OK;
    Temp t(c, c->buf_bytes);
    if (!t.p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes (the in-place state read back)", t.bytes);
    CK(enqueue_aa_gather(c, t.p), "gather launch");
    SweepArgs a = sweep_args(c, 0);
    a.src = t.p;
    a.dst = c->buf[0];
    CK(launch_sweep_aa(a, 3, c->stream), "store swapped");
    CK(enqueue_aa_prepare(c), "prepare pressure links");
    CK(cudaStreamSynchronize(c->stream), "normalize");
    c->aa_phase = 0;
    return LBM_OK;
}

int ensure_event(lbm_ctx *c, size_t idx)
{
    while (c->ev.size() <= idx) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e), "cudaEventCreate");
        c->ev.push_back(e);
    }
    return LBM_OK;
}

int direct_steps(lbm_ctx *c, int n)
{
    for (int s = 0; s < n; ++s) {
        if (c->aa) {
            const int ph = c->aa_phase;
            if (c->profiling) {
                // exchange interval: the forward exchange; the reverse
                // exchange is timed with the sweep
                size_t base = c->ev_used;
                int rc = ensure_event(c, base + 2);
                if (rc) return rc;
                const bool has_x = ph == 0 && !c->aa_fwd.empty();
                CK(cudaEventRecord(c->ev[base], c->stream), "cudaEventRecord");
                if (has_x) CK(enqueue_aa_fwd(c), "exchange launch");
                CK(cudaEventRecord(c->ev[base + 1], c->stream), "cudaEventRecord");
                CK(enqueue_aa_sweep(c, ph == 0 ? 1 : 0), "sweep launch");
                if (ph == 0) CK(enqueue_aa_rev(c), "exchange launch");
                CK(cudaEventRecord(c->ev[base + 2], c->stream), "cudaEventRecord");
                c->ev_has_x.push_back(has_x ? 1 : 0);
                c->ev_used += 3;
            } else {
                CK(enqueue_aa_step(c, ph), "step launch");
            }
            c->aa_phase ^= 1;
            continue;
        }
        if (c->profiling) {
            size_t base = c->ev_used;
            int rc = ensure_event(c, base + 2);
            if (rc) return rc;
            const bool has_x = exchange_each_step(c);
            CK(cudaEventRecord(c->ev[base], c->stream), "cudaEventRecord");
            if (has_x) CK(enqueue_exchange(c, c->cur), "exchange launch");
            CK(cudaEventRecord(c->ev[base + 1], c->stream), "cudaEventRecord");
            CK(enqueue_sweep(c, c->cur), "sweep launch");
            CK(cudaEventRecord(c->ev[base + 2], c->stream), "cudaEventRecord");
            c->ev_has_x.push_back(has_x ? 1 : 0);
            c->ev_used += 3;
        } else {
            CK(enqueue_step(c, c->cur), "step launch");
        }
        c->cur ^= 1;
    }
    return LBM_OK;
}

int ensure_graph(lbm_ctx *c, int par)
{
    if (c->graph[par]) return LBM_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int from = par;
    cudaError_t le = cudaSuccess;
    for (int s = 0; s < c->graph_steps && le == cudaSuccess; ++s) {
        le = enqueue_step(c, from);
        from ^= 1;
    }
    cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, le, "launch during capture");
    }
    if (ee != cudaSuccess) return cuda_fail(c, ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(&c->graph[par], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        c->graph[par] = nullptr;
        return cuda_fail(c, ie, "graph instantiate");
    }
    return LBM_OK;
}

int reduce(lbm_ctx *c, bool with_prev, std::vector<double> &out)
{
    int rc0 = check_device_error(c);
    if (rc0) return rc0;
    FieldArgs a = field_args(c);
    std::unique_ptr<Temp> t;
    const void *st = nullptr;
    if (with_prev && c->aa) return fail(c, LBM_EINVAL, "in-place streaming keeps no previous state");
    if ((rc0 = readable_state(c, t, &st, a))) return rc0;
    CK(launch_reduce(a, st, with_prev ? c->buf[c->cur ^ 1] : nullptr, c->d_partial, c->d_inst_begin, c->ninst,
                     c->d_red, c->stream),
       "reduce launch");
    out.assign(size_t(R_K) * c->ninst, 0.0);
    CK(cudaMemcpyAsync(out.data(), c->d_red, sizeof(double) * out.size(), cudaMemcpyDeviceToHost,
                       c->stream),
       "reduce D2H");
    CK(cudaStreamSynchronize(c->stream), "reduce sync");
    return LBM_OK;
}

std::string tune_key(const lbm_ctx *c)
{
    std::ostringstream k;
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    k << prop.name << "|st" << c->storage << "|c" << c->p.collision << "|f" << int(c->forced)
      << "|n" << c->blocks.size();
    // the block shapes (sorted) describe the work
    std::vector<std::string> shapes;
    for (const BlockGeom &b : c->blocks) {
        std::ostringstream s;
        s << b.nx << "x" << b.ny << "x" << b.nz;
        shapes.push_back(s.str());
    }
    std::sort(shapes.begin(), shapes.end());
    size_t h = 1469598103934665603ull;
    for (auto &s : shapes)
        for (char ch : s) h = (h ^ size_t(uint8_t(ch))) * 1099511628211ull;
    k << "|h" << std::hex << h;
    return k.str();
}

}  // namespace

// Message reported by lbm_last_error(NULL) for entry points without a context.
void lbm::set_global_error(const char *msg) { g_create_error = msg ? msg : ""; }

// =================================================================== C ABI
extern "C" {

void lbm_default_params(lbm_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->collision = LBM_BGK;
    p->magic = 3.0 / 16.0;
    p->rho0 = 1.0;
    for (int f = 0; f < 6; ++f) p->face_bc[f] = LBM_NOSLIP;
    p->storage = LBM_F32;
    p->storage_scale = 1.0;
    p->stream = nullptr;
    p->graph_steps = 0;
}

static int create_common(const std::vector<InstSpec> &inst, const lbm_params *pin, lbm_ctx **out)
{
    if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_params p;
    if (pin)
        p = *pin;
    else
        lbm_default_params(&p);
    if (!validate_params(p))
        return fail(nullptr, LBM_EINVAL, "invalid lbm_params (collision, storage, rho0, magic, "
                    "face_bc or storage_scale out of range)");
    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "out of host memory");
    c->p = p;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->alloc = g_alloc;
    }
    int rc;
    try {
        rc = build_context(c, inst);
    } catch (const std::bad_alloc &) {
        rc = fail(c, LBM_ENOMEM, "out of host memory");
    }
    if (rc != LBM_OK) {
        g_create_error = c->err;
        lbm_destroy(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

int lbm_create(const int dims[3], const int block_dims[3], double tau, const uint8_t *flags,
               const lbm_params *p, lbm_ctx **out)
{
    if (out) *out = nullptr;
    if (!dims || !block_dims) return fail(nullptr, LBM_EINVAL, "dims and block_dims are required");
    InstSpec s{};
    for (int a = 0; a < 3; ++a) {
        if (dims[a] <= 0 || block_dims[a] <= 0 || dims[a] % block_dims[a] != 0)
            return fail(nullptr, LBM_EINVAL,
                        "dims[%d]=%d must be a positive multiple of block_dims[%d]=%d", a, dims[a],
                        a, block_dims[a]);
        s.dims[a] = dims[a];
        s.bdims[a] = block_dims[a];
    }
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, LBM_EINVAL, "tau must be > 1/2");
    s.tau = tau;
    s.flags = flags;
    return create_common({s}, p, out);
}

int lbm_batch_create(int n, const int *dims, const double *tau, const uint8_t *const *flags,
                     const lbm_params *p, lbm_ctx **out)
{
    if (out) *out = nullptr;
    if (n <= 0 || !dims || !tau) return fail(nullptr, LBM_EINVAL, "n > 0, dims and tau are required");
    std::vector<InstSpec> inst(n);
    for (int k = 0; k < n; ++k) {
        for (int a = 0; a < 3; ++a) {
            if (dims[3 * k + a] <= 0)
                return fail(nullptr, LBM_EINVAL, "instance %d: dims must be positive", k);
            inst[k].dims[a] = inst[k].bdims[a] = dims[3 * k + a];
        }
        if (!(tau[k] > 0.5) || !std::isfinite(tau[k]))
            return fail(nullptr, LBM_EINVAL, "instance %d: tau must be > 1/2", k);
        inst[k].tau = tau[k];
        inst[k].flags = flags ? flags[k] : nullptr;
    }
    return create_common(inst, p, out);
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    invalidate_graphs(c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (auto it = c->owned.rbegin(); it != c->owned.rend(); ++it) dev_free(c, it->ptr, it->bytes);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbm_step(lbm_ctx *c, int n)
{
    if (!c || n < 0) return fail(c, LBM_EINVAL, "lbm_step: bad arguments");
    if (n == 0) return LBM_OK;
    int rc;
    if (c->profiling || c->graph_steps == 0) {
        rc = direct_steps(c, n);
    } else {
        rc = LBM_OK;
        if (c->aa && c->aa_phase == 1) {  // graphs start from the natural layout
            rc = direct_steps(c, 1);
            --n;
        }
        while (n >= c->graph_steps && rc == LBM_OK) {
            rc = ensure_graph(c, c->cur);
            if (rc) break;
            CK(cudaGraphLaunch(c->graph[c->cur], c->stream), "cudaGraphLaunch");
            n -= c->graph_steps;  // even: parity unchanged
        }
        if (rc == LBM_OK && n > 0) rc = direct_steps(c, n);
    }
    if (rc == LBM_OK) c->have_prev = true;
    return rc;
}

int lbm_synchronize(lbm_ctx *c)
{
    if (!c) return fail(c, LBM_EINVAL, "ctx is NULL");
    CK(cudaStreamSynchronize(c->stream), "lbm_synchronize");
    return check_device_error(c);
}

int lbm_macroscopic_device(lbm_ctx *c, float *rho, float *u)
{
    if (!c || !rho || !u) return fail(c, LBM_EINVAL, "lbm_macroscopic_device: NULL argument");
    std::unique_ptr<Temp> t;
    const void *st = nullptr;
    FieldArgs fa = field_args(c);
    int rc = readable_state(c, t, &st, fa);
    if (rc) return rc;
    CK(launch_macroscopic(fa, st, rho, u, c->stream), "macroscopic launch");
    if (t) CK(cudaStreamSynchronize(c->stream), "macroscopic");
    return LBM_OK;
}

int lbm_macroscopic(lbm_ctx *c, float *rho, float *u)
{
    if (!c || !rho || !u) return fail(c, LBM_EINVAL, "lbm_macroscopic: NULL argument");
    const size_t n = size_t(c->cells);
    Temp t(c, sizeof(float) * 4 * n);
    if (!t.p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes", t.bytes);
    float *dr = static_cast<float *>(t.p), *du = dr + n;
    int rc = lbm_macroscopic_device(c, dr, du);
    if (rc) return rc;
    CK(cudaMemcpyAsync(rho, dr, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream), "D2H rho");
    CK(cudaMemcpyAsync(u, du, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, c->stream), "D2H u");
    CK(cudaStreamSynchronize(c->stream), "lbm_macroscopic");
    return check_device_error(c);
}

int lbm_get_pdfs(lbm_ctx *c, double *f)
{
    if (!c || !f) return fail(c, LBM_EINVAL, "lbm_get_pdfs: NULL argument");
    const size_t n = size_t(c->cells) * Q;
    Temp t(c, sizeof(double) * n);
    if (!t.p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes", t.bytes);
    std::unique_ptr<Temp> g;
    const void *st = nullptr;
    FieldArgs fa = field_args(c);
    int rc = readable_state(c, g, &st, fa);
    if (rc) return rc;
    CK(launch_get_pdfs(fa, st, static_cast<double *>(t.p), c->stream), "get_pdfs launch");
    CK(cudaMemcpyAsync(f, t.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "D2H pdfs");
    CK(cudaStreamSynchronize(c->stream), "lbm_get_pdfs");
    return check_device_error(c);
}

int lbm_set_pdfs(lbm_ctx *c, const double *f)
{
    if (!c || !f) return fail(c, LBM_EINVAL, "lbm_set_pdfs: NULL argument");
    const size_t n = size_t(c->cells) * Q;
    Temp t(c, sizeof(double) * n);
    if (!t.p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes", t.bytes);
    CK(cudaMemcpyAsync(t.p, f, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "H2D pdfs");
    CK(launch_set_pdfs(write_args(c), c->buf[c->cur], static_cast<const double *>(t.p), c->stream),
       "set_pdfs launch");
    CK(enqueue_aa_prepare(c), "prepare pressure links");
    CK(cudaStreamSynchronize(c->stream), "lbm_set_pdfs");
    c->have_prev = false;
    c->aa_phase = 0;
    return LBM_OK;
}

int lbm_get_pdfs_device(lbm_ctx *c, double *f)
{
    if (!c || !f) return fail(c, LBM_EINVAL, "lbm_get_pdfs_device: NULL argument");
    std::unique_ptr<Temp> g;
    const void *st = nullptr;
    FieldArgs fa = field_args(c);
    int rc = readable_state(c, g, &st, fa);
    if (rc) return rc;
    CK(launch_get_pdfs(fa, st, f, c->stream), "get_pdfs launch");
    // an odd-time in-place state was read back into a transient array
    if (g) CK(cudaStreamSynchronize(c->stream), "lbm_get_pdfs_device");
    return LBM_OK;
}

int lbm_set_pdfs_device(lbm_ctx *c, const double *f)
{
    if (!c || !f) return fail(c, LBM_EINVAL, "lbm_set_pdfs_device: NULL argument");
    CK(launch_set_pdfs(write_args(c), c->buf[c->cur], f, c->stream), "set_pdfs launch");
    CK(enqueue_aa_prepare(c), "prepare pressure links");
    c->have_prev = false;
    c->aa_phase = 0;
    return LBM_OK;
}

int lbm_init_equilibrium_device(lbm_ctx *c, const float *rho, const float *u)
{
    if (!c || !rho || !u) return fail(c, LBM_EINVAL, "lbm_init_equilibrium_device: NULL argument");
    CK(launch_init_equilibrium(write_args(c), c->buf[c->cur], rho, u, c->stream), "init launch");
    CK(enqueue_aa_prepare(c), "prepare pressure links");
    c->have_prev = false;
    c->aa_phase = 0;
    return LBM_OK;
}

int lbm_init_equilibrium(lbm_ctx *c, const float *rho, const float *u)
{
    if (!c || !rho || !u) return fail(c, LBM_EINVAL, "lbm_init_equilibrium: NULL argument");
    const size_t n = size_t(c->cells);
    Temp t(c, sizeof(float) * 4 * n);
    if (!t.p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes", t.bytes);
    float *dr = static_cast<float *>(t.p), *du = dr + n;
    CK(cudaMemcpyAsync(dr, rho, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream), "H2D rho");
    CK(cudaMemcpyAsync(du, u, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c->stream), "H2D u");
    int rc = lbm_init_equilibrium_device(c, dr, du);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream), "lbm_init_equilibrium");
    return LBM_OK;
}

int lbm_invariants(lbm_ctx *c, double *mass, double mom[3], double *nonfinite, double *per_instance)
{
    if (!c) return fail(c, LBM_EINVAL, "ctx is NULL");
    std::vector<double> r;
    int rc = reduce(c, false, r);
    if (rc) return rc;
    const lbm_params &p = c->p;
    double M = 0, J[3] = {0, 0, 0}, bad = 0;
    for (int k = 0; k < c->ninst; ++k) {
        const double *v = &r[size_t(R_K) * k];
        const double m = v[R_NFLUID] * p.rho0 + v[R_DRHO];
        const double *F = &c->iforce[size_t(3 * k)];
        const double j[3] = {v[R_JX] - v[R_NFLUID] * 0.5 * F[0], v[R_JY] - v[R_NFLUID] * 0.5 * F[1],
                             v[R_JZ] - v[R_NFLUID] * 0.5 * F[2]};
        M += m;
        for (int a = 0; a < 3; ++a) J[a] += j[a];
        bad += v[R_NONFINITE];
        if (per_instance) {
            per_instance[5 * k] = m;
            for (int a = 0; a < 3; ++a) per_instance[5 * k + 1 + a] = j[a];
            per_instance[5 * k + 4] = v[R_NONFINITE];
        }
    }
    if (mass) *mass = M;
    if (mom)
        for (int a = 0; a < 3; ++a) mom[a] = J[a];
    if (nonfinite) *nonfinite = bad;
    return LBM_OK;
}

int lbm_residual(lbm_ctx *c, double *res, double *per_instance)
{
    if (!c || !res) return fail(c, LBM_EINVAL, "lbm_residual: NULL argument");
    if (c->aa)
        return fail(c, LBM_EINVAL, "lbm_residual: in-place streaming keeps no previous state (use "
                    "lbm_snapshot_velocity and lbm_residual_vs_snapshot, or lbm_run_to_residual)");
    if (!c->have_prev)
        return fail(c, LBM_EINVAL, "lbm_residual: no step has been taken since the state was set");
    std::vector<double> r;
    int rc = reduce(c, true, r);
    if (rc) return rc;
    double num = 0, den = 0;
    auto ratio = [](double a, double b) {
        if (b == 0.0) return a == 0.0 ? 0.0 : INFINITY;
        return std::sqrt(a) / std::sqrt(b);
    };
    for (int k = 0; k < c->ninst; ++k) {
        const double *v = &r[size_t(R_K) * k];
        num += v[R_DU2];
        den += v[R_U2];
        if (per_instance) per_instance[k] = ratio(v[R_DU2], v[R_U2]);
    }
    *res = ratio(num, den);
    return LBM_OK;
}

int lbm_run_to_residual(lbm_ctx *c, double tol, int check_every, long long max_steps,
                        long long *steps, double *res)
{
    if (!c || check_every <= 0 || max_steps < 0)
        return fail(c, LBM_EINVAL, "lbm_run_to_residual: bad arguments");
    long long done = 0;
    double r = INFINITY;
    while (done < max_steps) {
        const int n = int(std::min<long long>(check_every, max_steps - done));
        int rc;
        if (c->aa) {
            // the same one-step residual, against a velocity snapshot taken
            // one step before the end of the interval
            if (n > 1 && (rc = lbm_step(c, n - 1))) return rc;
            if ((rc = lbm_snapshot_velocity(c))) return rc;
            if ((rc = lbm_step(c, 1))) return rc;
            done += n;
            rc = lbm_residual_vs_snapshot(c, 1, &r, nullptr);
        } else {
            rc = lbm_step(c, n);
            if (rc) return rc;
            done += n;
            rc = lbm_residual(c, &r, nullptr);
        }
        if (rc) return rc;
        if (std::isnan(r)) {
            if (steps) *steps = done;
            if (res) *res = r;
            return fail(c, LBM_ENUMERIC, "residual is NaN after %lld steps", done);
        }
        if (r < tol) break;
    }
    if (steps) *steps = done;
    if (res) *res = r;
    return LBM_OK;
}

int lbm_impose_velocity_device(lbm_ctx *c, const float *u)
{
    if (!c || !u) return fail(c, LBM_EINVAL, "lbm_impose_velocity_device: NULL argument");
    int rc = aa_normalize(c);
    if (rc) return rc;
    CK(launch_impose_velocity(write_args(c), c->buf[c->cur], u, c->stream), "impose velocity");
    CK(enqueue_aa_prepare(c), "prepare pressure links");
    c->have_prev = false;
    return LBM_OK;
}

int lbm_init_consistent_device(lbm_ctx *c, const float *rho, const float *u, int iterations)
{
    if (!c || !rho || !u || iterations < 0) return fail(c, LBM_EINVAL, "lbm_init_consistent_device: bad arguments");
    int rc = lbm_init_equilibrium_device(c, rho, u);
    for (int k = 0; k < iterations && rc == LBM_OK; ++k) {
        if ((rc = lbm_step(c, 1))) break;
        rc = lbm_impose_velocity_device(c, u);
    }
    return rc;
}

int lbm_snapshot_velocity(lbm_ctx *c)
{
    if (!c) return fail(c, LBM_EINVAL, "ctx is NULL");
    if (!c->d_snap) {
        int rc = own(c, &c->d_snap, sizeof(float) * 4 * size_t(c->cells));
        if (rc) return rc;
    }
    std::unique_ptr<Temp> t;
    const void *st = nullptr;
    FieldArgs fa = field_args(c);
    int rc = readable_state(c, t, &st, fa);
    if (rc) return rc;
    CK(launch_macroscopic(fa, st, c->d_snap, c->d_snap + c->cells, c->stream), "snapshot");
    if (t) CK(cudaStreamSynchronize(c->stream), "snapshot");
    return LBM_OK;
}

int lbm_residual_vs_snapshot(lbm_ctx *c, int steps_since, double *res, double *per_instance)
{
    if (!c || !res || steps_since <= 0) return fail(c, LBM_EINVAL, "lbm_residual_vs_snapshot: bad arguments");
    if (!c->d_snap) return fail(c, LBM_EINVAL, "lbm_residual_vs_snapshot: no snapshot taken");
    int rc = check_device_error(c);
    if (rc) return rc;
    std::vector<double> r(size_t(R_K) * c->ninst, 0.0);
    std::unique_ptr<Temp> t;
    const void *st = nullptr;
    FieldArgs fa = field_args(c);
    if ((rc = readable_state(c, t, &st, fa))) return rc;
    CK(launch_reduce_snap(fa, st, c->d_snap + c->cells, c->d_partial, c->d_inst_begin,
                          c->ninst, c->d_red, c->stream),
       "snapshot residual");
    CK(cudaMemcpyAsync(r.data(), c->d_red, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, c->stream), "D2H");
    CK(cudaStreamSynchronize(c->stream), "sync");
    auto ratio = [&](double a, double b) {
        if (b == 0.0) return a == 0.0 ? 0.0 : INFINITY;
        return std::sqrt(a) / (std::sqrt(b) * double(steps_since));
    };
    double num = 0, den = 0;
    for (int k = 0; k < c->ninst; ++k) {
        const double *v = &r[size_t(R_K) * k];
        num += v[R_DU2];
        den += v[R_U2];
        if (per_instance) per_instance[k] = v[R_NONFINITE] > 0 ? NAN : ratio(v[R_DU2], v[R_U2]);
    }
    *res = ratio(num, den);
    return LBM_OK;
}

int lbm_set_forces(lbm_ctx *c, const double *force)
{
    if (!c || !force) return fail(c, LBM_EINVAL, "lbm_set_forces: NULL argument");
    for (int i = 0; i < 3 * c->ninst; ++i)
        if (!std::isfinite(force[i])) return fail(c, LBM_EINVAL, "lbm_set_forces: non-finite force");
    c->iforce.assign(force, force + 3 * c->ninst);
    bool forced = false;
    for (double f : c->iforce) forced |= f != 0.0;
    std::vector<char> consts = c->storage == LBM_F64 ? make_consts<double>(c) : make_consts<float>(c);
    if (consts.size() != c->h_consts.size()) return fail(c, LBM_EINVAL, "lbm_set_forces: constants size");
    CK(cudaStreamSynchronize(c->stream), "lbm_set_forces");
    CK(cudaMemcpy(c->d_consts, consts.data(), consts.size(), cudaMemcpyHostToDevice), "lbm_set_forces upload");
    c->h_consts.swap(consts);
    c->forced = forced;
    invalidate_graphs(c);
    return LBM_OK;
}

int lbm_run_to_residual_each(lbm_ctx *c, double tol, int check_every, int interval, long long max_steps,
                             long long *steps, double *res)
{
    if (!c || check_every <= 0 || max_steps < 0 || !steps || (interval && (check_every & 1)))
        return fail(c, LBM_EINVAL, "lbm_run_to_residual_each: bad arguments (interval residuals need an "
                    "even check_every)");
    if (c->aa || c->sparse)
        return fail(c, LBM_EINVAL, "lbm_run_to_residual_each: in-place streaming and the fluid-cell list "
                    "serve single Patches (use lbm_run_to_residual)");
    const int K = c->ninst;
    std::vector<double> r(size_t(K), INFINITY);
    // PDF range of each instance (its Blocks are contiguous)
    std::vector<long long> lo(size_t(K), -1), hi(size_t(K), 0);
    for (const BlockGeom &b : c->blocks) {
        if (lo[size_t(b.inst)] < 0) lo[size_t(b.inst)] = b.pdf_base;
        hi[size_t(b.inst)] = b.pdf_base + (long long)Q * b.G;
    }
    for (int k = 0; k < K; ++k) steps[k] = -1;
    c->active.assign(size_t(K), 1);
    int remaining = K, rc = LBM_OK;
    long long done = 0;
    if (interval && (rc = lbm_snapshot_velocity(c))) {
        c->active.clear();
        return rc;
    }
    while (remaining > 0 && done < max_steps) {
        const int n = int(std::min<long long>(check_every, max_steps - done));
        if ((rc = lbm_step(c, n))) break;
        done += n;
        double tot = 0;
        if (interval) {
            if ((rc = lbm_residual_vs_snapshot(c, n, &tot, r.data()))) break;
            if ((rc = lbm_snapshot_velocity(c))) break;
        } else if ((rc = lbm_residual(c, &tot, r.data()))) {
            break;
        }
        bool changed = false;
        for (int k = 0; k < K && rc == LBM_OK; ++k) {
            if (steps[k] >= 0) continue;
            if (std::isnan(r[size_t(k)])) {
                rc = fail(c, LBM_ENUMERIC, "instance %d: residual is NaN after %lld steps", k, done);
            } else if (r[size_t(k)] < tol) {
                // converged: keep its state in both buffers and stop sweeping it
                steps[k] = done;
                if (res) res[k] = r[size_t(k)];
                char *b0 = static_cast<char *>(c->buf[c->cur]), *b1 = static_cast<char *>(c->buf[c->cur ^ 1]);
                const size_t off = size_t(lo[size_t(k)]) * c->elem, len = size_t(hi[size_t(k)] - lo[size_t(k)]) * c->elem;
                CK(cudaMemcpyAsync(b1 + off, b0 + off, len, cudaMemcpyDeviceToDevice, c->stream), "freeze copy");
                c->active[size_t(k)] = 0;
                --remaining;
                changed = true;
            }
        }
        if (rc) break;
        if (changed && remaining > 0 && (rc = set_sweep(c, c->sw_tile, c->flat, c->grid))) break;
    }
    for (int k = 0; k < K; ++k)
        if (steps[k] < 0 && res) res[k] = r[size_t(k)];
    c->active.clear();
    const int rc2 = set_sweep(c, c->sw_tile, c->flat, c->grid);
    return rc ? rc : rc2;
}

// Clears every curved-wall distance of the context.
static int clear_wall_distances(lbm_ctx *c)
{
    if (c->has_curved) {
        CK(launch_curved_setup(nullptr, nullptr, nullptr, 0, c->d_flags, c->d_links, c->stored, c->d_curv_idx,
                               nullptr, c->stream),
           "curved clear");
        CK(cudaStreamSynchronize(c->stream), "curved clear");
        invalidate_graphs(c);
    }
    c->has_curved = false;
    c->curved_links = 0;
    return LBM_OK;
}

int lbm_set_wall_distances(lbm_ctx *c, long long n, const long long *cells, const int *dirs, const double *q)
{
    if (!c) return fail(c, LBM_EINVAL, "ctx is NULL");
    int rc0 = clear_wall_distances(c);  // a refused call leaves none set
    if (rc0) return rc0;
    if (n < 0 || (n > 0 && (!cells || !dirs || !q)))
        return fail(c, LBM_EINVAL, "lbm_set_wall_distances: bad arguments");
    if (c->aa || c->sparse)
        return fail(c, LBM_EINVAL, "lbm_set_wall_distances: in-place streaming and the fluid-cell list take no "
                    "curved walls");
    // each link: flag index of the fluid cell and of its pull source, table row
    const size_t nl = static_cast<size_t>(n);
    std::vector<long long> fidx(nl), sidx(nl);
    std::vector<int> rows(nl);
    std::unordered_map<long long, int> row_of;
    std::vector<int> first(size_t(c->ninst), -1);
    for (size_t bi = 0; bi < c->blocks.size(); ++bi)
        if (first[size_t(c->blocks[bi].inst)] < 0) first[size_t(c->blocks[bi].inst)] = int(bi);
    for (long long k = 0; k < n; ++k) {
        const long long cell = cells[k];
        const int d = dirs[k];
        if (cell < 0 || cell >= c->cells || d < 1 || d >= Q || !(q[k] > 0.0 && q[k] <= 1.0))
            return fail(c, LBM_EINVAL, "lbm_set_wall_distances: link %lld (cell %lld, direction %d, q %g) "
                        "out of range", k, cell, d, q[k]);
        const int inst = int(std::upper_bound(c->inst_out_base.begin(), c->inst_out_base.end(), cell) -
                             c->inst_out_base.begin()) - 1;
        const int *N = &c->idims[size_t(3 * inst)];
        const long long local = cell - c->inst_out_base[size_t(inst)];
        const int x = int(local % N[0]), y = int((local / N[0]) % N[1]), z = int(local / ((long long)N[0] * N[1]));
        const BlockGeom &b0 = c->blocks[size_t(first[size_t(inst)])];
        const int nbx = N[0] / b0.nx, nby = N[1] / b0.ny;
        const BlockGeom &b = c->blocks[size_t(first[size_t(inst)] + ((z / b0.nz) * nby + y / b0.ny) * nbx + x / b0.nx)];
        const long long pxyf = (long long)b.pxf * b.py;
        const long long cf = (z % b.nz + 1) * pxyf + (long long)(y % b.ny + 1) * b.pxf + x % b.nx + OXF;
        fidx[size_t(k)] = b.cell_base + cf;
        sidx[size_t(k)] = b.cell_base + cf - (ex(d) + ey(d) * (long long)b.pxf + ez(d) * pxyf);
        rows[size_t(k)] = row_of.emplace(fidx[size_t(k)], int(row_of.size())).first->second;
    }
    const size_t nrows = row_of.size();
    const bool f64 = c->storage == LBM_F64;
    const size_t tbytes = std::max<size_t>(nrows, 1) * 18 * (f64 ? 8 : 4);
    std::vector<char> table(tbytes);
    for (size_t r = 0; r < std::max<size_t>(nrows, 1) * 18; ++r) {
        if (f64)
            reinterpret_cast<double *>(table.data())[r] = 0.5;
        else
            reinterpret_cast<float *>(table.data())[r] = 0.5f;
    }
    for (long long k = 0; k < n; ++k) {
        const size_t at = size_t(rows[size_t(k)]) * 18 + size_t(dirs[k] - 1);
        if (f64)
            reinterpret_cast<double *>(table.data())[at] = q[k];
        else
            reinterpret_cast<float *>(table.data())[at] = float(q[k]);
    }
    disown(c, c->d_curv_q);
    c->d_curv_q = nullptr;
    int rc;
    if ((rc = upload(c, reinterpret_cast<char **>(&c->d_curv_q), table))) return rc;
    if (!c->d_curv_idx && (rc = own(c, &c->d_curv_idx, sizeof(int) * size_t(std::max<long long>(c->stored, 1)))))
        return rc;
    CK(cudaMemsetAsync(c->d_curv_idx, 0xff, sizeof(int) * size_t(c->stored), c->stream), "memset");
    Temp t(c, (sizeof(long long) * 2 + sizeof(int)) * size_t(std::max<long long>(n, 1)) + sizeof(int));
    if (!t.p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes", t.bytes);
    long long *dfi = static_cast<long long *>(t.p), *dsi = dfi + n;
    int *drows = reinterpret_cast<int *>(dsi + n), *dbad = drows + n;
    if (n > 0) {
        CK(cudaMemcpyAsync(dfi, fidx.data(), sizeof(long long) * size_t(n), cudaMemcpyHostToDevice, c->stream), "H2D");
        CK(cudaMemcpyAsync(dsi, sidx.data(), sizeof(long long) * size_t(n), cudaMemcpyHostToDevice, c->stream), "H2D");
        CK(cudaMemcpyAsync(drows, rows.data(), sizeof(int) * size_t(n), cudaMemcpyHostToDevice, c->stream), "H2D");
    }
    CK(cudaMemsetAsync(dbad, 0, sizeof(int), c->stream), "memset");
    CK(launch_curved_setup(dfi, dsi, drows, n, c->d_flags, c->d_links, c->stored, c->d_curv_idx, dbad, c->stream),
       "curved setup");
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "D2H");
    CK(cudaStreamSynchronize(c->stream), "lbm_set_wall_distances");
    invalidate_graphs(c);
    if (bad) {
        c->has_curved = true;  // bits may be set: clear them
        if ((rc = clear_wall_distances(c))) return rc;
        return fail(c, LBM_EINVAL, "lbm_set_wall_distances: %d link(s) do not start at a fluid cell or do not "
                    "pull from a resting wall (LBM_NOSLIP); no distances set", bad);
    }
    c->has_curved = n > 0;
    c->curved_links = n;
    if (c->has_curved) {  // the TMA sweep has no curved links
        c->kernel = LBM_KERNEL_REGISTER;
        c->tma_grid = 0;
    }
    return LBM_OK;
}

int lbm_get_info(lbm_ctx *c, lbm_info *info)
{
    if (!c || !info) return fail(c, LBM_EINVAL, "lbm_get_info: NULL argument");
    info->cells = c->cells;
    info->fluid_cells = c->fluid;
    info->stored_cells = c->stored;
    info->blocks = int(c->blocks.size());
    info->instances = c->ninst;
    info->storage = c->storage;
    info->bytes_per_pdf = c->elem;
    info->exchange_pdfs = c->exchange_pdfs;
    info->device_bytes = c->device_bytes;
    for (int a = 0; a < 3; ++a) info->tile[a] = c->sw_tile[a];
    info->tiles = (long long)c->stiles.size();
    info->kernel = c->kernel;
    info->stages = c->kernel == LBM_KERNEL_TMA ? tma_stages(c->storage) : 0;
    info->flat = c->kernel != LBM_KERNEL_TMA ? c->flat : 0;
    info->pair = c->kernel != LBM_KERNEL_TMA ? c->pair : 0;
    info->mask = c->kernel != LBM_KERNEL_TMA ? c->mask : 0;
    info->streaming = c->aa ? LBM_STREAM_AA : LBM_STREAM_TWO_GRID;
    info->aa_phase = c->aa_phase;
    info->layout = c->sparse ? LBM_LAYOUT_SPARSE : LBM_LAYOUT_BLOCKS;
    info->list_cells = c->nfluid;
    info->sweep_ctas = c->kernel == LBM_KERNEL_TMA ? c->tma_grid
                       : c->grid > 0                ? c->grid
                                                    : int(c->stiles.size());
    if (c->kernel == LBM_KERNEL_TMA) {
        info->tile[0] = c->blocks[0].nx;
        info->tile[1] = 256 / c->blocks[0].nx;
        info->tile[2] = c->tma_zchunk;
    }
    return LBM_OK;
}

int lbm_profile_enable(lbm_ctx *c, int on)
{
    if (!c) return fail(c, LBM_EINVAL, "ctx is NULL");
    c->profiling = on != 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx *c, lbm_profile *out)
{
    if (!c || !out) return fail(c, LBM_EINVAL, "lbm_profile_read: NULL argument");
    CK(cudaStreamSynchronize(c->stream), "profile sync");
    for (size_t s = 0; s * 3 < c->ev_used; ++s) {
        float x = 0.f, w = 0.f;
        CK(cudaEventElapsedTime(&x, c->ev[3 * s], c->ev[3 * s + 1]), "elapsed");
        CK(cudaEventElapsedTime(&w, c->ev[3 * s + 1], c->ev[3 * s + 2]), "elapsed");
        if (c->ev_has_x[s]) {
            c->acc_x_ms += x;
            ++c->acc_x;
        }
        c->acc_sweep_ms += w;
        ++c->acc_sweeps;
    }
    c->ev_used = 0;
    c->ev_has_x.clear();
    out->sweep_ms = c->acc_sweep_ms;
    out->sweep_launches = c->acc_sweeps;
    out->exchange_ms = c->acc_x_ms;
    out->exchange_launches = c->acc_x;
    c->acc_sweep_ms = c->acc_x_ms = 0;
    c->acc_sweeps = c->acc_x = 0;
    return LBM_OK;
}

namespace {

// Sweep configuration {kind, tx, ty, tz, grid, minb, zchunk, mask}: kind 0 =
// register sweep over row tiles, 1 = TMA sweep, 2 = register sweep over runs
// of tx consecutive cells.
int check_cfg(lbm_ctx *c, const int *cd)
{
    const bool tma_ok = c->kernel == LBM_KERNEL_TMA || (c->tma_grid > 0);
    if (cd[0] < 0 || cd[0] > 4) return fail(c, LBM_EINVAL, "sweep config: kind %d", cd[0]);
    if (cd[0] == 1 && !tma_ok)
        return fail(c, LBM_EINVAL, "sweep config: the TMA sweep does not apply to this context");
    if (c->aa && (cd[0] == 1 || cd[7] != 0))
        return fail(c, LBM_EINVAL, "sweep config: in-place streaming takes the register sweep with near-wall "
                    "cells by lane (kinds 0, 2, 3, 4; mask 0)");
    if (cd[0] >= 3) {
        bool even = c->storage != LBM_F64;
        for (const BlockGeom &b : c->blocks) even = even && (b.nx % 2 == 0);
        if (!even)
            return fail(c, LBM_EINVAL, "sweep config: two cells per thread need even Block widths and "
                        "FP32 / F16S / BF16S storage");
    }
    if ((cd[0] == 2 || cd[0] == 4) && (cd[1] < 32 || cd[1] > 256 || cd[1] % 32 != 0))
        return fail(c, LBM_EINVAL, "sweep config: runs of %d threads (32..256, multiple of 32)", cd[1]);
    if ((cd[0] == 0 || cd[0] == 3) &&
        (cd[1] <= 0 || cd[2] <= 0 || cd[3] <= 0 || cd[1] % 32 != 0 || cd[1] * cd[2] > 256))
        return fail(c, LBM_EINVAL, "sweep config: tile %dx%dx%d", cd[1], cd[2], cd[3]);
    if (cd[0] == 1 && (cd[6] <= 0 || cd[6] > 1024)) return fail(c, LBM_EINVAL, "sweep config: zchunk %d", cd[6]);
    if (cd[4] < 0) return fail(c, LBM_EINVAL, "sweep config: grid %d", cd[4]);
    if (cd[5] != 3 && cd[5] != 4) return fail(c, LBM_EINVAL, "sweep config: minb %d (3 or 4)", cd[5]);
    if (cd[7] != 0 && cd[7] != 1) return fail(c, LBM_EINVAL, "sweep config: mask %d", cd[7]);
    return LBM_OK;
}

int apply_cfg(lbm_ctx *c, const int *cd)
{
    int rc = check_cfg(c, cd);
    if (rc) return rc;
    // the TMA sweep keeps the current register work list (used if switched back)
    const int t[3] = {cd[0] == 1 ? c->sw_tile[0] : cd[1], cd[0] == 1 ? c->sw_tile[1] : cd[2],
                      cd[0] == 1 ? c->sw_tile[2] : cd[3]};
    const int flat = (cd[0] == 2 || cd[0] == 4) ? cd[1] : (cd[0] == 1 ? c->flat : 0);
    const int pair = cd[0] >= 3 ? 1 : (cd[0] == 1 ? c->pair : 0);
    if ((rc = set_sweep(c, t, flat, cd[0] == 1 ? c->grid : cd[4], pair))) return rc;
    c->minb = cd[5];
    if (cd[0] == 1) c->tma_zchunk = cd[6];
    c->mask = cd[7];
    c->kernel = cd[0] == 1 ? LBM_KERNEL_TMA : LBM_KERNEL_REGISTER;
    invalidate_graphs(c);
    return LBM_OK;
}

void get_cfg(const lbm_ctx *c, int *cd)
{
    cd[0] = c->kernel == LBM_KERNEL_TMA ? 1 : (c->flat > 0 ? (c->pair ? 4 : 2) : (c->pair ? 3 : 0));
    cd[1] = c->sw_tile[0];
    cd[2] = c->sw_tile[1];
    cd[3] = c->sw_tile[2];
    cd[4] = c->grid;
    cd[5] = c->minb;
    cd[6] = c->tma_zchunk;
    cd[7] = c->mask;
}

}  // namespace

int lbm_get_sweep_config(lbm_ctx *c, int cfg[8])
{
    if (!c || !cfg) return fail(c, LBM_EINVAL, "lbm_get_sweep_config: NULL argument");
    get_cfg(c, cfg);
    return LBM_OK;
}

int lbm_set_sweep_config(lbm_ctx *c, const int cfg[8])
{
    if (!c || !cfg) return fail(c, LBM_EINVAL, "lbm_set_sweep_config: NULL argument");
    return apply_cfg(c, cfg);
}

int lbm_autotune(lbm_ctx *c, const char *cache_path, int best_out[3])
{
    if (!c) return fail(c, LBM_EINVAL, "ctx is NULL");
    const bool tma_ok = c->kernel == LBM_KERNEL_TMA || (c->tma_grid > 0);
    const std::string key = tune_key(c) + (tma_ok ? "|tma" : "") + (c->aa ? "|aa" : "") + (c->sparse ? "|list" : "");
    // configuration: kind (0 register sweep over row tiles, 1 TMA sweep, 2
    // register sweep over runs of tx consecutive cells), tx, ty, tz, grid,
    // minb, zchunk, mask
    using Cfg = std::array<int, 8>;
    Cfg best;
    get_cfg(c, best.data());
    const int kind0 = best[0];
    bool cached = false;
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        const std::string needle = "\"key\": \"" + key + "\"";
        while (std::getline(in, line)) {
            if (line.find(needle) == std::string::npos) continue;
            size_t t = line.find("\"cfg\": [");
            Cfg v;
            if (t != std::string::npos &&
                std::sscanf(line.c_str() + t, "\"cfg\": [%d, %d, %d, %d, %d, %d, %d, %d]", &v[0], &v[1],
                            &v[2], &v[3], &v[4], &v[5], &v[6], &v[7]) == 8) {
                best = v;
                cached = true;
            }
        }
    }
    auto apply = [&](const Cfg &cd) -> int { return apply_cfg(c, cd.data()); };
    if (!cached) {
        const char *ev = std::getenv("LBM_AUTOTUNE_VERBOSE");
        const bool verbose = ev && ev[0] == '1';
        int maxnx = 0;
        for (const BlockGeom &b : c->blocks) maxnx = std::max(maxnx, b.nx);
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int zc0 = c->tma_zchunk, m0 = c->mask;
        bool pair_ok = c->storage != LBM_F64;
        for (const BlockGeom &b : c->blocks) pair_ok = pair_ok && (b.nx % 2 == 0);
        const int *st = c->sw_tile;
        std::vector<Cfg> cand;
        if (c->sparse) {  // the list sweep: register budget and grid only
            for (int mb : {3, 4})
                for (int m : {0, 4, 8, 16}) cand.push_back({0, st[0], st[1], st[2], m * sms, mb, zc0, 0});
        }
        if (tma_ok)
            for (int zc : {2, 4, 8, 16, 32}) cand.push_back({1, st[0], st[1], st[2], 0, c->minb, zc, m0});
        for (int mb : {3, 4}) {
            if (c->sparse) break;
            for (int tx : {32, 64, 128, 256}) {
                if (tx > std::max(32, round_up(maxnx, 32))) continue;
                for (int th : {128, 256}) {
                    if (th < tx) continue;
                    for (int tz : {1, 2, 4, 8}) cand.push_back({0, tx, th / tx, tz, 0, mb, zc0, m0});
                }
            }
            for (int th : {128, 256}) cand.push_back({2, th, 1, 1, 0, mb, zc0, m0});
            if (pair_ok) {
                // two cells per thread: row tiles of 2 tx cells, runs of 2 th cells
                for (int tx : {32, 64}) {
                    if (tx > std::max(32, round_up((maxnx + 1) / 2, 32))) continue;
                    for (int th : {128, 256}) {
                        if (th < tx) continue;
                        for (int tz : {1, 2, 4}) cand.push_back({3, tx, th / tx, tz, 0, mb, zc0, m0});
                    }
                }
                for (int th : {128, 256}) cand.push_back({4, th, 1, 1, 0, mb, zc0, m0});
            }
        }
        // persistent grids over the default work list
        for (int m : {4, 8, 16}) if (!c->sparse)
            cand.push_back({kind0 == 1 ? 0 : kind0, st[0], st[1], st[2], m * sms, c->minb, zc0, m0});
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        // in place the timed steps change the state: it is saved here and
        // restored after tuning (a transient second array)
        std::unique_ptr<Temp> saved;
        if (c->aa) {
            int rc = aa_normalize(c);
            if (rc) return rc;
            saved.reset(new Temp(c, c->buf_bytes));
            if (!saved->p) return fail(c, LBM_ENOMEM, "temporary of %zu bytes (state saved while tuning)",
                                      saved->bytes);
            CK(cudaMemcpyAsync(saved->p, c->buf[0], c->buf_bytes, cudaMemcpyDeviceToDevice, c->stream), "save");
        }
        auto time_cfg = [&](const Cfg &cd, int reps, float *ms_out) -> int {
            int rc = apply(cd);
            if (rc) return rc;
            if (c->aa) {  // pairs of steps: the local one and the odd one with its exchanges
                CK(enqueue_aa_step(c, 0), "tune");
                CK(enqueue_aa_step(c, 1), "tune");
                CK(cudaEventRecord(e0, c->stream), "event");
                for (int r = 0; r < reps; ++r) {
                    CK(enqueue_aa_step(c, 0), "tune");
                    CK(enqueue_aa_step(c, 1), "tune");
                }
                CK(cudaEventRecord(e1, c->stream), "event");
                CK(cudaEventSynchronize(e1), "tune sync");
                float ms = 0;
                CK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
                *ms_out = ms / (2 * reps);
                return LBM_OK;
            }
            CK(enqueue_sweep(c, c->cur), "tune");
            CK(cudaEventRecord(e0, c->stream), "event");
            for (int r = 0; r < reps; ++r) CK(enqueue_sweep(c, c->cur), "tune");
            CK(cudaEventRecord(e1, c->stream), "event");
            CK(cudaEventSynchronize(e1), "tune sync");
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            *ms_out = ms / reps;
            if (verbose)
                std::fprintf(stderr,
                             "lbm_autotune: %s tile %d %d %d grid %d minb %d zchunk %d mask %d: %.4f ms/sweep"
                             " (%d reps)\n",
                             cd[0] == 1 ? "tma" : (cd[0] == 2 ? "flat" : "rows"), cd[1], cd[2], cd[3], cd[4],
                             cd[5], cd[6], cd[7], *ms_out, reps);
            return LBM_OK;
        };
        // pass 1: every candidate, briefly
        std::vector<std::pair<float, Cfg>> timed;
        for (const Cfg &cd : cand) {
            float ms = 0;
            int rc = time_cfg(cd, 5, &ms);
            if (rc) return rc;
            timed.push_back({ms, cd});
        }
        std::sort(timed.begin(), timed.end(),
                  [](const std::pair<float, Cfg> &x, const std::pair<float, Cfg> &y) { return x.first < y.first; });
        // pass 2: the four fastest with both near-wall strategies, longer
        std::vector<Cfg> fin;
        for (size_t k = 0; k < timed.size() && k < 4; ++k) {
            Cfg cd = timed[k].second;
            fin.push_back(cd);
            if (cd[0] != 1 && !c->aa && !c->sparse) {
                cd[7] ^= 1;
                fin.push_back(cd);
            }
        }
        float best_ms = 1e30f;
        for (const Cfg &cd : fin) {
            float ms = 0;
            int rc = time_cfg(cd, 20, &ms);
            if (rc) return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best = cd;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (saved) {
            CK(cudaMemcpyAsync(c->buf[0], saved->p, c->buf_bytes, cudaMemcpyDeviceToDevice, c->stream),
               "restore");
            CK(cudaStreamSynchronize(c->stream), "restore");
        }
        int rc = check_device_error(c);
        if (rc) return rc;
        if (cache_path) {
            std::ofstream o(cache_path, std::ios::app);
            o << "{\"key\": \"" << key << "\", \"cfg\": [" << best[0];
            for (int k = 1; k < 8; ++k) o << ", " << best[k];
            o << "], \"ms_per_sweep\": " << best_ms << "}\n";
        }
    }
    int rc = apply(best);
    if (rc) return rc;
    c->have_prev = false;  // the scratch buffer was overwritten
    if (best_out)
        for (int a = 0; a < 3; ++a) best_out[a] = best[1 + a];
    CK(cudaStreamSynchronize(c->stream), "autotune");
    return LBM_OK;
}

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn release, void *user)
{
    if ((alloc == nullptr) != (release == nullptr))
        return fail(nullptr, LBM_EINVAL, "alloc and release must both be given or both be NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = release;
    g_alloc.user = user;
    return LBM_OK;
}

int lbm_directions(int *e, double *w, int *o)
{
    for (int q = 0; q < Q; ++q) {
        if (e) {
            e[3 * q] = ex(q);
            e[3 * q + 1] = ey(q);
            e[3 * q + 2] = ez(q);
        }
        if (w) w[q] = wq(q);
        if (o) o[q] = opp(q);
    }
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *c)
{
    if (c) return c->err.c_str();
    return g_create_error.c_str();
}

const char *lbm_version(void) { return "lbm 0.1 sm_103a"; }

}  // extern "C"
