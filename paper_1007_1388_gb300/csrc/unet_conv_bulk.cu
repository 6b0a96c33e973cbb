// Bulk-copy tensor-core 3x3x3 convolutions of the U-Net over planar tensors
// (layout in unet_internal.h).  In the planar layout every run of positions
// of one 8-channel group is contiguous, so operand tiles are 1-D bulk copies
// (cp.async.bulk) instead of tensor-map boxes, and a tap is a constant offset.
// Bulk copies complete about 3000 cycles after they are issued and cost tens
// to hundreds of cycles each to issue, so both kernels keep 150-220 KB per SM
// in flight in few, large copies.
//
// Convolution (persistent, one CTA per SM): a work item is `tiles` x 128
// consecutive positions q0.. of one grid's interior planes.  Per 16 input
// channels (one ring stage) the producer copies, for dz = -1, 0, 1, the run
// of positions [q0 + dz sz - sy - 1, + L) of both 8-channel groups: the slab
// every tap of that plane reaches.  The A operand of tap (dz, dy, dx) and tile
// i is the dz slab at position offset i 128 + (dy + 1) sy + dx + 1: K-major,
// no swizzle, rows (positions) 16 bytes apart (SBO 128), the two channel
// groups L 16 bytes apart (LBO); so 27 taps share one copy of their input.
// Weights stay resident when they fit (else they ride with every stage).  An
// M = 128 MMA costs max(46, N / 2) cycles whatever the operand layout
// (measured), so the 27 MMAs of N = cout per tile and stage run the tensor
// core near that rate as long as the epilogue keeps up: two epilogue warp
// groups take alternate work items, each with its own TMEM accumulator
// buffer, while the MMAs of the next item run.  Positions in halo columns and
// rows are computed and dropped.
//
// Weight gradient: each 16-row unit (tap, 16 input channels) of the 128-row
// tile and each 8-channel group of dy is a run of `run` positions (256, or
// 128 where two such stages do not fit), copied by the lanes of the
// producer warp; the MN-major operands have LBO 128 (8 positions) and SBO
// run x 16 bytes (8 channels).  K runs over every position of
// the grids, so dy comes with zeros at all non-interior positions.
//
// Every wait is bounded (2e9 cycles); a thread that gives up sets the error
// word and stops, the others time out in turn, every issued copy is awaited
// (bounded) before the CTA leaves, and every thread reaches the TMEM release.
#include "lbm_internal.h"
#include "umma.cuh"
#include "unet_internal.h"

namespace lbm {
namespace {

constexpr int CTHREADS = 320;  // warp 0: copies, warp 1: MMAs, warps 2-5 and 6-9: two epilogue groups
constexpr int CSTAGES = 3;
constexpr int WTHREADS = 128;
constexpr int WSTAGES = 4;  // weight-gradient ring depth, at most
constexpr int WRUN = 256;  // positions per weight-gradient stage, at most
constexpr long long kWait = 2000000000ll;
constexpr int kSmemBudget = 220 * 1024;

struct ConvPlan {
    int L;         // positions per dz slab (a multiple of 8)
    int slab;      // bytes of the three slabs of both 8-channel groups
    int wstage;    // bytes of one stage's weights
    int resident;  // all weights loaded once
    int wres;      // bytes of the resident weights (0 if not)
    int stage;     // bytes of one ring stage
    int nstages;   // ring depth
    int bufcols;   // TMEM columns of one accumulator buffer (tiles x cout)
    int nbuf;      // accumulator buffers: 2, or 1 where two do not fit TMEM
    int tcols;     // TMEM columns allocated (a power of two)
    int smem;      // dynamic shared memory
};

__host__ __device__ inline ConvPlan conv_plan(const VGrid &g, int cin, int cout, int tiles)
{
    ConvPlan c;
    const int sy = (1 << g.lx) + 2;
    c.L = (128 * tiles + 2 * sy + 2 + 7) / 8 * 8;
    c.slab = 3 * 2 * c.L * 16;
    c.wstage = 27 * 2 * cout * 16;
    const int wall = (cin / 16) * c.wstage;
    c.resident = wall <= 64 * 1024;
    c.wres = c.resident ? wall : 0;
    c.stage = c.slab + (c.resident ? 0 : c.wstage);
    const int n = (kSmemBudget - c.wres) / c.stage;
    c.nstages = n < CSTAGES ? n : CSTAGES;
    c.bufcols = tiles * cout;
    c.nbuf = 2 * c.bufcols <= 512 ? 2 : 1;
    c.tcols = 32;
    while (c.tcols < c.nbuf * c.bufcols) c.tcols <<= 1;
    c.smem = c.wres + c.nstages * c.stage;
    return c;
}

__device__ __forceinline__ const bf16 *group_base(const bf16 *s0, const bf16 *s1, int g0, int grp, long long ptot)
{
    return grp < g0 ? s0 + (long long)grp * ptot * 8 : s1 + (long long)(grp - g0) * ptot * 8;
}

template <int T>
__global__ void __launch_bounds__(CTHREADS, 1) conv3_bulk_kernel(const __grid_constant__ ConvBulkArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[CSTAGES], empty[CSTAGES], tfull[2], tempty[2], wbar;
    __shared__ uint32_t tslot;
    __shared__ int s_ok[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin = a.c0 + a.c1, cout = a.cout, nks = cin >> 4, g0 = a.c0 >> 3;
    const ConvPlan cp = conv_plan(a.g, cin, cout, T);
    const Planar P = planar_of(a.g);
    const int nx = 1 << a.g.lx, ny = 1 << a.g.ly, nz = 1 << a.g.lz;
    const int span = 128 * T;                            // output positions per work item
    const int tpg = int((nz * P.sz + span - 1) / span);  // work items per grid
    const int items = tpg * a.g.nb;
    unsigned char *wsm = smem;             // resident weights
    unsigned char *ring = smem + cp.wres;  // ring stages

    if (warp == 0) umma::tmem_alloc(&tslot, uint32_t(cp.tcols));
    if (tid == 0) {
        for (int s = 0; s < CSTAGES; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&tfull[b], 1);
            umma::mbar_init(&tempty[b], 4);
        }
        umma::mbar_init(&wbar, 1);
        umma::mbar_fence_init();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;

    if (tid == 0) {
        // producer
        if (cp.resident) {
            umma::mbar_arrive_expect_tx(&wbar, uint32_t(cp.wres));
            umma::bulk_load(wsm, a.w, uint32_t(cp.wres), &wbar);
        }
        int j = 0;
        bool ok = true;
        for (int item = blockIdx.x; ok && item < items; item += gridDim.x) {
            const int b = item / tpg;
            const long long q0 = P.guard + b * P.pg + P.sz + (long long)(item - b * tpg) * span;
            for (int k = 0; k < nks; ++k, ++j) {
                const int s = j % cp.nstages;
                if (j >= cp.nstages && !umma::mbar_wait(&empty[s], ((j / cp.nstages) - 1) & 1, kWait)) {
                    atomicExch(a.err, 1);
                    ok = false;
                    break;
                }
                unsigned char *st = ring + s * cp.stage;
                umma::mbar_arrive_expect_tx(&full[s], uint32_t(cp.stage));
                for (int dz = 0; dz < 3; ++dz)
                    for (int h = 0; h < 2; ++h) {
                        const bf16 *src = group_base(a.src0, a.src1, g0, 2 * k + h, P.ptot);
                        const long long q = q0 + (dz - 1) * P.sz - P.sy - 1;
                        umma::bulk_load(st + (dz * 2 + h) * cp.L * 16, src + q * 8, uint32_t(cp.L * 16), &full[s]);
                    }
                if (!cp.resident)
                    umma::bulk_load(st + cp.slab, a.w + (long long)k * 27 * 2 * cout * 8, uint32_t(cp.wstage),
                                    &full[s]);
            }
        }
        // before leaving: the copies of the last stages have landed (bounded)
        const int last = j < cp.nstages ? j : cp.nstages;
        for (int u = j - last; u < j; ++u) umma::mbar_wait(&full[u % cp.nstages], (u / cp.nstages) & 1, kWait);
        if (cp.resident) umma::mbar_wait(&wbar, 0, kWait);
    } else if (tid == 32) {
        // MMA issuer: per stage, 27 taps x T tiles, N = cout.  Row r of tile i
        // is position q0 + 128 i + r, at slab offset 128 i + r + (dy + 1) sy +
        // dx + 1.  Descriptors are built once per stage; a tap or tile moves
        // only the start address field (16-byte units, no carry out of its 14
        // bits: shared memory stays below 256 KB).  The packed weights hold the
        // three x taps of a (dz, dy) pair side by side: tap (pair, d) starts d
        // cout rows in, its two channel groups 3 cout rows apart (LBO).
        const uint32_t idesc = umma::idesc_bf16(cout, false, false);
        bool ok = !cp.resident || umma::mbar_wait(&wbar, 0, kWait);
        if (!ok) atomicExch(a.err, 1);
        int j = 0, it = 0;
        for (int item = blockIdx.x; ok && item < items; item += gridDim.x, ++it) {
            const int buf = cp.nbuf == 2 ? (it & 1) : 0, use = cp.nbuf == 2 ? (it >> 1) : it;
            if (use >= 1 && !umma::mbar_wait(&tempty[buf], (use - 1) & 1, kWait)) {
                atomicExch(a.err, 1);
                ok = false;
                break;
            }
            umma::fence_after();
            const uint32_t acc = tmem + uint32_t(buf * cp.bufcols);
            for (int k = 0; k < nks; ++k, ++j) {
                const int s = j % cp.nstages;
                if (!umma::mbar_wait(&full[s], (j / cp.nstages) & 1, kWait)) {
                    atomicExch(a.err, 1);
                    ok = false;
                    break;
                }
                umma::fence_after();
                const uint32_t base = umma::smem_addr(ring + s * cp.stage);
                const uint32_t wb = cp.resident ? umma::smem_addr(wsm) + uint32_t(k * cp.wstage) : base + uint32_t(cp.slab);
                const uint64_t a0 = umma::sdesc(base, uint32_t(cp.L * 16), 128);
                const uint64_t b0 = umma::sdesc(wb, uint32_t(3 * cout * 16), 128);
#pragma unroll
                for (int pr = 0; pr < 9; ++pr) {
                    const int dz = pr / 3, dy = pr - 3 * dz;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const uint64_t ad = a0 + uint64_t(dz * 2 * cp.L + dy * int(P.sy) + d);
                        const uint64_t bd = b0 + uint64_t(pr * 6 * cout + d * cout);
                        const uint32_t accumulate = (k > 0 || pr > 0 || d > 0) ? 1u : 0u;
#pragma unroll
                        for (int i = 0; i < T; ++i)
                            umma::mma_bf16(acc + uint32_t(i * cout), ad + uint64_t(i * 128), bd, idesc, accumulate);
                    }
                }
                umma::mma_commit(&empty[s]);
            }
            if (ok) umma::mma_commit(&tfull[buf]);
        }
    } else if (warp >= 2) {
        // epilogue: two groups of four warps take alternate work items (one
        // accumulator buffer each; with a single buffer group 0 takes all).
        // Warp w holds rows 32 (w % 4) .. + 31 of every tile.
        const int grp = (warp - 2) >> 2, quarter = warp & 3, r = quarter * 32 + lane;
        const uint32_t trow = tmem + (uint32_t(quarter * 32) << 16);
        const int barid = 1 + grp;
        int it = 0;
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
            const int buf = cp.nbuf == 2 ? (it & 1) : 0, use = cp.nbuf == 2 ? (it >> 1) : it;
            if ((cp.nbuf == 2 ? buf : 0) != grp) continue;
            // one thread waits for the group and shares the outcome, so that its
            // four warps leave together
            if ((warp & 3) == 2 && lane == 0) s_ok[grp] = umma::mbar_wait(&tfull[buf], use & 1, kWait) ? 1 : 0;
            asm volatile("bar.sync %0, 128;" ::"r"(barid) : "memory");
            const int ok = s_ok[grp];
            asm volatile("bar.sync %0, 128;" ::"r"(barid) : "memory");  // s_ok read before its next write
            if (!ok) {
                if ((warp & 3) == 2 && lane == 0) atomicExch(a.err, 1);
                break;
            }
            umma::fence_after();
            const int b = item / tpg;
            const long long q0 = P.guard + b * P.pg + P.sz + (long long)(item - b * tpg) * span;
            // position of row r in tile 0, then stepped by 128 per tile
            int rel = int(q0 - P.guard - b * P.pg) + r;
            int zp = rel / int(P.sz), rem = rel - zp * int(P.sz);
            int yp = rem / int(P.sy), xp = rem - yp * int(P.sy);
            for (int i = 0; i < T; ++i) {
                if (i > 0) {
                    xp += 128;
                    while (xp >= int(P.sy)) xp -= int(P.sy), ++yp;
                    while (yp >= ny + 2) yp -= ny + 2, ++zp;
                }
                const long long q = q0 + i * 128 + r;
                const bool out = zp >= 1 && zp <= nz && yp >= 1 && yp <= ny && xp >= 1 && xp <= nx;
                // the voxel's periodic copies (positions) and its unpadded index
                const long long dxh = xp == 1 ? nx : (xp == nx ? -nx : 0);
                const long long dzh = zp == 1 ? nz * P.sz : (zp == nz ? -nz * P.sz : 0);
                const long long m = (((long long)b * nz + zp - 1) * ny + yp - 1) * nx + xp - 1;
                const uint32_t col = trow + uint32_t(buf * cp.bufcols + i * cout);
                for (int c = 0; c < cout; c += 16) {
                    float v[16];
                    umma::tmem_ld16(col + uint32_t(c), v);  // warp-collective
                    if (!out) continue;
                    if (a.bias) {
                        const float4 *bb = reinterpret_cast<const float4 *>(a.bias + c);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float4 t4 = __ldg(bb + e);
                            v[4 * e] += t4.x, v[4 * e + 1] += t4.y, v[4 * e + 2] += t4.z, v[4 * e + 3] += t4.w;
                        }
                    }
                    if (a.relu)
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] = fmaxf(v[e], 0.f);
                    if (a.out_f32) {
                        float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(a.out) + m * cout + c);
#pragma unroll
                        for (int e = 0; e < 4; ++e) o[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                    } else {
                        __align__(16) __nv_bfloat162 h[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) h[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                        const uint4 w0 = reinterpret_cast<const uint4 *>(h)[0];
                        const uint4 w1 = reinterpret_cast<const uint4 *>(h)[1];
                        bf16 *o0 = static_cast<bf16 *>(a.out) + (long long)(c >> 3) * P.ptot * 8;
                        bf16 *o1 = o0 + P.ptot * 8;
                        const long long at[4] = {q, q + dxh, q + dzh, q + dxh + dzh};
                        const bool use4[4] = {true, dxh != 0, dzh != 0, dxh != 0 && dzh != 0};
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (use4[u]) {
                                *reinterpret_cast<uint4 *>(o0 + at[u] * 8) = w0;
                                *reinterpret_cast<uint4 *>(o1 + at[u] * 8) = w1;
                            }
                    }
                }
            }
            umma::fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&tempty[buf]);
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, uint32_t(cp.tcols));
}

template <int RUN>
__global__ void __launch_bounds__(WTHREADS, 1) wgrad_bulk_kernel(const __grid_constant__ WgradBulkArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[WSTAGES], empty[WSTAGES], done;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin = a.c0 + a.c1, cout = a.cout, g0 = a.c0 >> 3, NS = a.stages;
    constexpr int run = RUN, slot = RUN * 16;  // 8 channels x run positions
    const int abytes = 16 * slot, sbytes = abytes + (cout >> 3) * slot;
    uint32_t tcols = 32;
    while (tcols < uint32_t(cout)) tcols <<= 1;
    const Planar P = planar_of(a.g);
    const long long total = (long long)a.g.nb * P.pg;  // K: positions [guard, guard + total)
    const long long pbeg = (long long)blockIdx.y * a.pps;
    const long long pend = pbeg + a.pps < total ? pbeg + a.pps : total;
    const int nchunks = pend > pbeg ? int((pend - pbeg + run - 1) / run) : 0;
    const int row0 = blockIdx.x * 128;
    int units = (27 * cin - row0) / 16;  // 16-row units of this tile holding (tap, channel) rows
    units = units < 0 ? 0 : (units > 8 ? 8 : units);
    const int slots = 2 * units + (cout >> 3);

    if (warp == 0) umma::tmem_alloc(&tslot, tcols);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        umma::mbar_init(&done, 1);
        umma::mbar_fence_init();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = tslot;

    if (warp == 0) {
        // producer warp: one 4 KB run per slot, one slot per lane
        int c = 0;
        for (; c < nchunks; ++c) {
            const int s = c % NS;
            int ok = 1;
            if (lane == 0 && c >= NS && !umma::mbar_wait(&empty[s], ((c / NS) - 1) & 1, kWait)) ok = 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(a.err, 1);
                break;
            }
            if (lane == 0) umma::mbar_arrive_expect_tx(&full[s], uint32_t(slots * slot));
            __syncwarp();
            unsigned char *st = smem + s * sbytes;
            const long long q = P.guard + pbeg + (long long)c * run;
            for (int sl = lane; sl < slots; sl += 32) {
                if (sl < 2 * units) {
                    const int row = row0 + (sl >> 1) * 16;
                    const int t = row / cin, grp = ((row - t * cin) >> 3) + (sl & 1);
                    const long long off = (long long)(t / 9 - 1) * P.sz + ((t / 3) % 3 - 1) * P.sy + (t % 3 - 1);
                    const bf16 *src = group_base(a.src0, a.src1, g0, grp, P.ptot);
                    umma::bulk_load(st + sl * slot, src + (q + off) * 8, uint32_t(slot), &full[s]);
                } else {
                    const int grp = sl - 2 * units;
                    umma::bulk_load(st + abytes + grp * slot, a.dyz + ((long long)grp * P.ptot + q) * 8,
                                    uint32_t(slot), &full[s]);
                }
            }
        }
        // before leaving: the copies of the last stages have landed (bounded)
        if (lane == 0) {
            const int last = c < NS ? c : NS;
            for (int u = c - last; u < c; ++u) umma::mbar_wait(&full[u % NS], (u / NS) & 1, kWait);
        }
    } else if (tid == 32) {
        const uint32_t idesc = umma::idesc_bf16(cout, true, true);
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % NS;
            if (!umma::mbar_wait(&full[s], (c / NS) & 1, kWait)) {
                atomicExch(a.err, 1);
                ok = false;
                break;
            }
            umma::fence_after();
            const uint32_t sa = umma::smem_addr(smem + s * sbytes), sb = sa + uint32_t(abytes);
#pragma unroll
            for (int j = 0; j < run / 16; ++j)
                umma::mma_bf16(tmem, umma::sdesc(sa + j * 256, 128, uint32_t(slot)),
                               umma::sdesc(sb + j * 256, 128, uint32_t(slot)), idesc, (c > 0 || j > 0) ? 1u : 0u);
            umma::mma_commit(&empty[s]);
        }
        if (ok && nchunks > 0) umma::mma_commit(&done);
    }
    __syncwarp();
    const bool ready = nchunks > 0 && umma::mbar_wait(&done, 0, kWait);
    if (!ready && nchunks > 0 && tid == 0) atomicExch(a.err, 1);
    if (ready) umma::fence_after();
    const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
    const long long prow = (long long)blockIdx.y * a.rows_pad + row0 + tid;
    for (int c = 0; c < cout; c += 16) {
        float r[16];
        if (ready) {
            umma::tmem_ld16(trow + c, r);
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) r[e] = 0.f;
        }
        float4 *o = reinterpret_cast<float4 *>(a.partial + prow * cout + c);
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = make_float4(r[4 * e], r[4 * e + 1], r[4 * e + 2], r[4 * e + 3]);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, tcols);
}

// dw[co][t][ci] = sum over splits (in split order) of partial[split][t cin + ci][co]
__global__ void wgrad_bulk_reduce_kernel(const float *__restrict__ partial, int nsplit, int rows, int rows_pad,
                                         int cout, int cin, float *__restrict__ dw)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cout) return;
    const int r = int(i / cout), co = int(i - (long long)r * cout);
    float acc = 0.f;
    for (int s = 0; s < nsplit; ++s) acc += partial[((long long)s * rows_pad + r) * cout + co];
    const int t = r / cin, ci = r - t * cin;
    dw[((long long)co * 27 + t) * cin + ci] = acc;
}

size_t wgrad_bulk_smem(int cout, int run, int stages) { return size_t(stages) * (16 + (cout >> 3)) * run * 16; }

cudaError_t raise_smem_limit(const void *fn, size_t bytes, size_t &current)
{
    if (bytes <= current) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e == cudaSuccess) current = bytes;
    return e;
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

}  // namespace

size_t conv3_bulk_smem(const VGrid &g, int cin, int cout, int tiles)
{
    const ConvPlan c = conv_plan(g, cin, cout, tiles);
    return c.nstages >= 1 && c.tcols <= 512 ? size_t(c.smem) : ~size_t(0);
}

int conv3_bulk_buffers(const VGrid &g, int cin, int cout, int tiles) { return conv_plan(g, cin, cout, tiles).nbuf; }

int conv3_bulk_stages(const VGrid &g, int cin, int cout, int tiles) { return conv_plan(g, cin, cout, tiles).nstages; }

int wgrad_bulk_splits(const VGrid &g, int pps)
{
    const long long total = (long long)g.nb * planar_of(g).pg;
    return pps > 0 ? int((total + pps - 1) / pps) : 0;
}

// Two stages of the longest runs that fit: on GB300 fewer, larger copies beat
// a deeper ring of the same bytes (measured: 256 x 2 stages 3.03 ms per U-Net
// training step, 128 x 4 stages 4.02 ms, 128 x 3 stages 3.34 ms).
void wgrad_bulk_config(int cout, int *run, int *stages)
{
    int r = WRUN;
    while (r > 64 && wgrad_bulk_smem(cout, r, 2) > size_t(kSmemBudget)) r >>= 1;
    *run = r;
    *stages = 2;
}

int wgrad_bulk_pps(const VGrid &g, int row_tiles, int run)
{
    // about two waves of one CTA per SM
    const long long total = (long long)g.nb * planar_of(g).pg;
    long long nsplit = (2ll * sm_count() + row_tiles - 1) / row_tiles;
    if (nsplit < 1) nsplit = 1;
    long long pps = (total + nsplit - 1) / nsplit;
    pps = (pps + run - 1) / run * run;
    return int(pps);
}

cudaError_t launch_conv3_bulk(const ConvBulkArgs &a, cudaStream_t s)
{
    const int cin = a.c0 + a.c1;
    if (a.c0 <= 0 || a.c0 % 16 || a.c1 < 0 || a.c1 % 16 || (a.c1 && !a.src1) || !a.src0 || !a.w || !a.out ||
        a.cout <= 0 || a.cout % 16 || a.cout > 256 || a.tiles < 1 || a.tiles > 4 || a.g.lx < 1 || a.g.ly < 1 ||
        a.g.lz < 1 || a.g.lx > 8 || a.g.nb < 1 || planar_of(a.g).ptot >= (1ll << 31) ||
        (reinterpret_cast<uintptr_t>(a.bias) & 15))
        return cudaErrorInvalidValue;
    const size_t sm = conv3_bulk_smem(a.g, cin, a.cout, a.tiles);
    if (sm > size_t(kSmemBudget)) return cudaErrorInvalidValue;
    const void *fn = a.tiles == 4 ? reinterpret_cast<const void *>(conv3_bulk_kernel<4>)
                     : a.tiles == 2 ? reinterpret_cast<const void *>(conv3_bulk_kernel<2>)
                                    : reinterpret_cast<const void *>(conv3_bulk_kernel<1>);
    if (a.tiles != 1 && a.tiles != 2 && a.tiles != 4) return cudaErrorInvalidValue;
    static size_t current[3] = {0, 0, 0};
    cudaError_t e = raise_smem_limit(fn, sm, current[a.tiles >> 1]);
    if (e != cudaSuccess) return e;
    const Planar P = planar_of(a.g);
    const long long span = 128ll * a.tiles;
    const long long items = ((1ll << a.g.lz) * P.sz + span - 1) / span * a.g.nb;
    const long long grid = items < sm_count() ? items : sm_count();
    if (a.tiles == 4)
        conv3_bulk_kernel<4><<<unsigned(grid), CTHREADS, sm, s>>>(a);
    else if (a.tiles == 2)
        conv3_bulk_kernel<2><<<unsigned(grid), CTHREADS, sm, s>>>(a);
    else
        conv3_bulk_kernel<1><<<unsigned(grid), CTHREADS, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_wgrad_bulk(const WgradBulkArgs &a, int nsplit, float *dw, cudaStream_t s)
{
    const int cin = a.c0 + a.c1;
    if (a.c0 <= 0 || a.c0 % 16 || a.c1 < 0 || a.c1 % 16 || (a.c1 && !a.src1) || !a.src0 || !a.dyz || !dw ||
        !a.partial || a.cout <= 0 || a.cout % 16 || a.cout > 128 || a.run < 16 || a.run > WRUN || a.run % 16 ||
        a.stages < 1 || a.stages > WSTAGES || a.pps <= 0 || a.pps % a.run ||
        wgrad_bulk_smem(a.cout, a.run, a.stages) > size_t(kSmemBudget) ||
        a.rows_pad < 27 * cin || a.rows_pad % 128 || nsplit != wgrad_bulk_splits(a.g, a.pps) || a.g.lx < 1 ||
        a.g.ly < 1 || a.g.lz < 1 || a.g.lx > 8 || planar_of(a.g).ptot >= (1ll << 31))
        return cudaErrorInvalidValue;
    if (a.run != 64 && a.run != 128 && a.run != 256) return cudaErrorInvalidValue;
    const void *fn = a.run == 256 ? reinterpret_cast<const void *>(wgrad_bulk_kernel<256>)
                     : a.run == 128 ? reinterpret_cast<const void *>(wgrad_bulk_kernel<128>)
                                    : reinterpret_cast<const void *>(wgrad_bulk_kernel<64>);
    static size_t current[3] = {0, 0, 0};
    const size_t sm = wgrad_bulk_smem(a.cout, a.run, a.stages);
    cudaError_t e = raise_smem_limit(fn, sm, current[a.run == 256 ? 2 : (a.run == 128 ? 1 : 0)]);
    if (e != cudaSuccess) return e;
    const dim3 grid(unsigned(a.rows_pad / 128), unsigned(nsplit));
    if (nsplit > 0) {
        if (a.run == 256)
            wgrad_bulk_kernel<256><<<grid, WTHREADS, sm, s>>>(a);
        else if (a.run == 128)
            wgrad_bulk_kernel<128><<<grid, WTHREADS, sm, s>>>(a);
        else
            wgrad_bulk_kernel<64><<<grid, WTHREADS, sm, s>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = 27ll * cin * a.cout;
    wgrad_bulk_reduce_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(a.partial, nsplit, 27 * cin, a.rows_pad,
                                                                         a.cout, cin, dw);
    return cudaGetLastError();
}

}  // namespace lbm
