// Sweep configurations of the host runtime (lbm_get/set_sweep_config) and
// the autotuner (lbm_autotune): which register or TMA sweep, tile,
// register budget, persistent grid and near-wall strategy a context runs,
// chosen by timing candidates on the GPU and cached per device and workload.
#include "ctx_internal.h"

using namespace lbm;
using namespace lbm::rt;

namespace {

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

// Sweep configuration {kind, tx, ty, tz, grid, minb, zchunk, mask}: kind 0 =
// register sweep over row tiles, 1 = TMA sweep, 2 = register sweep over runs
// of tx consecutive cells; 3 / 4 = 0 / 2 with two cells per thread.
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
    if (cd[5] != 3 && cd[5] != 4 && cd[5] != 5) return fail(c, LBM_EINVAL, "sweep config: minb %d (3, 4 or 5)", cd[5]);
    if (cd[5] == 5 && ((cd[0] != 0 && cd[0] != 2) || c->aa || c->sparse || c->storage == LBM_F64))
        return fail(c, LBM_EINVAL, "sweep config: minb 5 applies to the one-cell register sweep (kinds 0 and 2) "
                    "of two-array Block layouts with FP32 / F16S / BF16S storage");
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

extern "C" {

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
            for (int zc : {2, 4, 8, 16, 32}) cand.push_back({1, st[0], st[1], st[2], 0, std::min(c->minb, 4), zc, m0});
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
            if (mb == 4 && !c->aa && c->storage != LBM_F64) {  // 48 registers, one cell per thread
                for (int th : {128, 256}) cand.push_back({2, th, 1, 1, 0, 5, zc0, m0});
                for (int tx : {32, 64})
                    if (tx <= std::max(32, round_up(maxnx, 32))) cand.push_back({0, tx, 128 / tx, 2, 0, 5, zc0, m0});
            }
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
        for (int m : {4, 8, 16})
            if (!c->sparse)
                cand.push_back({kind0 == 1 ? 0 : kind0, st[0], st[1], st[2], m * sms,
                                kind0 == 0 || kind0 == 2 ? c->minb : std::min(c->minb, 4), zc0, m0});
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

}  // extern "C"
