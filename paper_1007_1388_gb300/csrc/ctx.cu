// Host runtime of liblbm.so: contexts, device memory, the launch helpers
// (exchange, sweep, CUDA-graph replay of time steps, launch timing) and the
// C ABI of include/lbm.h.  The context builder (Patch/Block layout, flags,
// exchange plans) is in ctx_build.cu, the sweep configurations and the
// autotuner in ctx_tune.cu.
//
// A context holds one Patch split into Blocks (Sec. 4.2), or a batch of
// independent single-Block instances.  All Blocks of all instances live in
// two device buffers (src / dst, Sec. 2.1 two-grid pull scheme), each Block
// with a one-cell ghost shell.  One time step is one Sweep (Sec. 4): the
// communication step (exchange kernel, device memory only; the local
// "buffer swap" of Sec. 4.4 becomes a direct ghost-layer copy) followed by the
// work step (sweep kernel over every Block in one launch).
#include "ctx_internal.h"

using namespace lbm;
using namespace lbm::rt;

namespace lbm {
namespace rt {

Allocator g_alloc;
thread_local std::string g_create_error;
std::mutex g_alloc_mu;

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
    // A single instance's collision constants reach the kernel as parameters,
    // except in the one-cell 16-bit sweep with link masks, which measured
    // faster reading them from global memory (one sphere-packed 256x256x128
    // channel, F16S: 0.244 against 0.304 ms per sweep; FP32 and the two-cell
    // sweeps are faster with parameters)
    const bool narrow = c->storage == LBM_F16S || c->storage == LBM_BF16S;
    const bool onecell = c->kernel == LBM_KERNEL_REGISTER && !c->aa && !c->sparse && !c->pair;
    a.unif = c->ninst == 1 && !(narrow && onecell && c->mask) ? 1 : 0;
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

cudaError_t enqueue_aa_sweep(const lbm_ctx *c, int mode, void *gather_dst)
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

}  // namespace rt
}  // namespace lbm

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

// Message reported by lbm_last_error(NULL) for entry points without a context.
void lbm::set_global_error(const char *msg) { lbm::rt::g_create_error = msg ? msg : ""; }

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
        if (changed && remaining > 0 && (rc = set_sweep(c, c->sw_tile, c->flat, c->grid, c->pair))) break;
    }
    for (int k = 0; k < K; ++k)
        if (steps[k] < 0 && res) res[k] = r[size_t(k)];
    c->active.clear();
    const int rc2 = set_sweep(c, c->sw_tile, c->flat, c->grid, c->pair);
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
