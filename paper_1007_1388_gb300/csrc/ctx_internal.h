// Internals of the host runtime shared by its translation units: the
// context (struct lbm_ctx, opaque in the C ABI), device memory ownership,
// error reporting, the context builder, the launch helpers and the tuner's
// configuration.  Not part of the C ABI.
#pragma once

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

namespace lbm {
namespace rt {

struct Allocator {
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn release = nullptr;
    void *user = nullptr;
};

struct DevMem {
    void *ptr = nullptr;
    size_t bytes = 0;
};

extern Allocator g_alloc;
extern thread_local std::string g_create_error;
extern std::mutex g_alloc_mu;

}  // namespace rt
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
    std::vector<lbm::BlockGeom> blocks;
    std::vector<lbm::Tile> tiles;
    std::vector<long long> inst_tile_begin;
    std::vector<lbm::XSlab> xslabs;
    std::vector<long long> inst_out_base;
    long long cells = 0, fluid = 0, stored = 0, exchange_pdfs = 0;
    int tile[3] = {64, 4, 4};     // tiles of the field and reduction kernels (fixed at create)
    // the sweep's own work list (lbm_autotune changes only this)
    int sw_tile[3] = {64, 4, 4};  // row tile, or {flat, 1, 1}
    int flat = 0;                 // > 0: runs of this many consecutive cells per CTA
    int grid = 0;                 // 0 = one CTA per tile, else a persistent grid
    int mask = 0;                 // near-wall cells via link masks under a warp vote
    int pair = 0;                 // two neighbouring cells per thread (FP32 / 16-bit storage)
    std::vector<lbm::Tile> stiles;
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
    std::vector<lbm::XSlabF> aa_fwd;   // ghost rows <- neighbours' boundary rows, before the odd step
    std::vector<lbm::XSlabF> aa_rev;   // neighbours' boundary rows <- ghost rows, after it
    lbm::XSlabF *d_aa_fwd = nullptr;
    lbm::XSlabF *d_aa_rev = nullptr;
    // fluid-cell list layout (LBM_LAYOUT_SPARSE): list index per flag cell,
    // neighbour table [19][nstride]
    bool sparse = false;
    long long nfluid = 0, nstride = 0;
    int *d_sidx = nullptr;
    int *d_nbr = nullptr;
    // kernel choice and the TMA sweep's launch state
    int kernel = LBM_KERNEL_REGISTER;
    lbm::TmaMaps maps{};
    int tma_zchunk = 8;
    int tma_grid = 0;
    int *d_err = nullptr;       // device error word written by timed-out waits
    // device
    lbm::rt::Allocator alloc;
    std::vector<lbm::rt::DevMem> owned;
    void *buf[2] = {nullptr, nullptr};
    uint8_t *d_flags = nullptr;
    uint32_t *d_links = nullptr;
    lbm::BlockGeom *d_blocks = nullptr;
    lbm::Tile *d_tiles = nullptr;
    lbm::Tile *d_stiles = nullptr;
    lbm::XSlab *d_xslabs = nullptr;
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

namespace lbm {
namespace rt {

// ---- errors and device memory (ctx.cu)
int fail(lbm_ctx *c, int code, const char *fmt, ...);
int cuda_fail(lbm_ctx *c, cudaError_t e, const char *what);
void *dev_alloc(lbm_ctx *c, size_t bytes);
void dev_free(lbm_ctx *c, void *p, size_t bytes);
void disown(lbm_ctx *c, void *p);

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

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

// ---- the context builder (ctx_build.cu)
// Instance description used while building a context.
struct InstSpec {
    int dims[3];
    int bdims[3];
    double tau;
    const uint8_t *flags;
};

int round_up(int v, int a);
long long plane_cells(long long cells, int elem);
uint8_t classify(const lbm_params &p, const int N[3], const uint8_t *flags, long long X, long long Y, long long Z);
void build_tiles(lbm_ctx *c, const int t[3], std::vector<Tile> &tiles, std::vector<long long> &begin);
int validate_params(const lbm_params &p);
template <typename T>
std::vector<char> make_consts(const lbm_ctx *c);
void invalidate_graphs(lbm_ctx *c);
int set_tiles(lbm_ctx *c, const int t[3]);
int set_sweep(lbm_ctx *c, const int t[3], int flat, int grid, int pair);
bool tma_applicable(const lbm_ctx *c);
int setup_tma(lbm_ctx *c);
int build_context(lbm_ctx *c, const std::vector<InstSpec> &inst);

// ---- launches (ctx.cu)
SweepArgs sweep_args(const lbm_ctx *c, int from);
FieldArgs field_args(const lbm_ctx *c);
FieldArgs write_args(const lbm_ctx *c);
cudaError_t enqueue_exchange(const lbm_ctx *c, int which);
cudaError_t enqueue_sweep(const lbm_ctx *c, int from);
bool exchange_each_step(const lbm_ctx *c);
cudaError_t enqueue_aa_fwd(const lbm_ctx *c);
cudaError_t enqueue_aa_rev(const lbm_ctx *c);
cudaError_t enqueue_aa_sweep(const lbm_ctx *c, int mode, void *gather_dst = nullptr);
cudaError_t enqueue_aa_step(const lbm_ctx *c, int ph);
cudaError_t enqueue_step(const lbm_ctx *c, int from);
int check_device_error(lbm_ctx *c);
cudaError_t enqueue_aa_prepare(const lbm_ctx *c);
cudaError_t enqueue_aa_gather(const lbm_ctx *c, void *dst);
int readable_state(lbm_ctx *c, std::unique_ptr<Temp> &t, const void **state, FieldArgs &fa);
int aa_normalize(lbm_ctx *c);
int ensure_event(lbm_ctx *c, size_t idx);
int direct_steps(lbm_ctx *c, int n);
int ensure_graph(lbm_ctx *c, int par);
int reduce(lbm_ctx *c, bool with_prev, std::vector<double> &out);

}  // namespace rt
}  // namespace lbm
