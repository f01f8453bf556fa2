// roeam_api.cu — host implementation of the C ABI declared in include/roeam.h.
//
// Owns the device memory of a batch of grids, lays the state out as pitched
// structure-of-arrays planes, drives the fused stage kernels (directly or through a
// cached CUDA graph of several steps), and runs the FP64 monitor reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "roeam.h"
#include "roeam_internal.h"

using namespace roeam;

namespace {

thread_local std::string g_last_error;

roeam_status fail(roeam_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                                      \
    do {                                                                                                    \
        cudaError_t e_ = (expr);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? ROEAM_E_OOM : ROEAM_E_CUDA, "%s: %s (%s:%d)", #expr, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                        \
    } while (0)

long long round_up(long long a, long long m) { return (a + m - 1) / m * m; }

constexpr int GRAPH_STEPS = 8;   // SSP-RK3 steps per captured graph (an even number)

// NVTX range around a library call (visible in a profiler's timeline; free without one).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Autotuner results of this process, by workload (see tune_key).
struct TuneResult { int best; double ms[NUM_TILE_CFGS]; };
std::mutex g_tune_mu;
std::map<std::string, TuneResult> g_tune_cache;
constexpr size_t MAX_GRAPHS = 8; // captured graphs kept per handle (one per (cfl, dt_fixed) pair)

struct GraphKey {
    double cfl, dt_fixed;
    bool operator<(const GraphKey &o) const { return cfl < o.cfl || (cfl == o.cfl && dt_fixed < o.dt_fixed); }
};

}  // namespace

struct roeam_grid {
    int device = 0;
    cudaStream_t stream = nullptr;       // user stream (work is ordered on it)
    cudaStream_t cap_stream = nullptr;   // private stream used only for graph capture
    // roeam_step_host: streams for the copies in, the computation and the copies out, and
    // events (the start, then two per chunk: copied in, computed)
    cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> pipe_ev;
    // roeam_step_host's own unit table: each chunk's units, cut so that the chunk alone gives
    // every resident warp a unit (rebuilt when the chunks or the tile shape change)
    int4 *d_units_pipe = nullptr;
    int pipe_units_cap = 0, pipe_cfg = -1;
    std::vector<std::pair<int, int>> pipe_chunks;
    std::vector<int> pipe_tile_base;
    int precision = 32, muscl = 0, curv = 0, kind = KIND_PLAIN, count = 0;   // kind: StageKind
    size_t esize = 4;
    int tile_cfg = 0;
    int eff_ty = 0, eff_dyn = 0;    // the current shape's segment height (after halving) and schedule
    int nblocks = 0;        // persistent CTAs of the stage kernel
    int num_sms = 0;
    long long total_elems = 0, total_vert = 0, total_packed = 0, total_solid = 0;
    int max_cells = 0;
    int total_tiles = 0;
    std::vector<GridDev> hg;
    std::vector<int> h_tile_base;
    std::vector<char> state_set;
    GridDev *d_grids = nullptr;
    void *d_coef = nullptr;                              // GridCoef<T>[count]
    int4 *d_units_grid = nullptr;   // work units grouped by grid (per-grid launches)
    int4 *d_units_all = nullptr;    // the same units ordered by decreasing size (whole-batch launches)
    int4 *d_units_part = nullptr;   // interior units (by decreasing size), then the EXCHANGE edge units
    int part_split = 0;             // first edge unit in d_units_part
    int part_next = 0;              // 1: the interior part of stage stage_next ran, its edges are due
    int units_cap = 0;
    void *U = nullptr, *A = nullptr, *B = nullptr;      // U^n (in place), stage buffers
    void *vdx = nullptr, *vdy = nullptr;
    uint8_t *solid = nullptr;
    int stage_next = 0;              // next stage of a step run stage by stage (roeam_rk_stage)
    double *staging = nullptr;
    unsigned long long *rate = nullptr;                  // 2 x count slots (double bits)
    unsigned *status = nullptr;
    unsigned *work = nullptr;                            // dynamic unit-scheduling counters (2)
    double *partials = nullptr;
    int partial_rows = 0;
    double *red_out = nullptr;                           // 8 doubles
    double *h_red = nullptr;                             // pinned 8 doubles
    unsigned long long *h_rate = nullptr;                // pinned count
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;     // ordering against a caller's stream (device-pointer I/O)
    long long step = 0;
    unsigned long long launches = 0;
    std::map<GraphKey, cudaGraphExec_t> graphs;
};

// roeam_step_host cuts the batch into chunks of whole grids with about these shares of the
// cells: the first and the last chunks are small, so that the copies out start early and the
// copies in end early, and both directions of the host link are busy together for most of the
// step (measured against eight equal chunks: 2.85 against 2.95 ms per step on the 512-grid
// batch with float32 host arrays).
static const double PIPE_SHARES[] = {1, 2, 3, 4, 4, 4, 4, 3, 2, 1};

// Shortest segment height the halving below goes to (a grid's segments differ by at most one
// row, so where its rows do not divide evenly some come out one row shorter).
constexpr int MIN_SEGMENT_ROWS = 2;

namespace {

// Work units of the stage kernel for shape `cfg`: every grid is cut into strips of
// 32 - 2H interior columns and into ceil(nj / ty) segments of nearly equal height. A batch
// too small to give every resident warp a unit (a single grid of a few thousand cells, like
// the paper's test cases) gets shorter segments, down to MIN_SEGMENT_ROWS: each segment
// re-reads H + 1 rows above its first, but the rows are swept by many more warps at once. Units are stored
// grouped by grid (for launches over one grid) and, for whole-batch launches, ordered by
// decreasing height so that the static round-robin over warps stays balanced.
roeam_status setup_tiles(roeam_grid *g, int cfg)
{
    const TileCfg tc = TILE_CFGS[cfg];
    g->tile_cfg = cfg;
    const int H = g->muscl ? 2 : 1;
    const int width = tc.tx - 2 * H;
    const int occ = g->precision == 32 ? Launchers<float>::stage_occupancy(g->muscl, g->curv, g->kind)
                                       : Launchers<double>::stage_occupancy(g->muscl, g->curv, g->kind);
    const long long warps = (long long)std::max(1, occ) * g->num_sms;
    int ty = tc.ty;
    for (;;) {
        long long units = 0;
        for (const GridDev &G : g->hg) units += (long long)((G.ni + width - 1) / width) * ((G.nj + ty - 1) / ty);
        if (units >= warps || ty <= MIN_SEGMENT_ROWS) break;
        const int next = std::max(MIN_SEGMENT_ROWS, ty / 2);
        if (next < 4) {
            // Below 4 rows a unit re-reads about as many warm-up rows as it writes: halve there
            // only while the units still fit one round of the resident warps (a single grid's
            // segment count may drop by an eighth below to make them fit). The 400^2 corner's
            // 2-row units took two rounds and stepped slower than its 4-row ones.
            long long fit = 0;
            for (const GridDev &G : g->hg) {
                const long long nty = (G.nj + next - 1) / next;
                fit += (long long)((G.ni + width - 1) / width) * (g->count == 1 ? nty - nty / 8 : nty);
            }
            if (fit > warps) break;
        }
        ty = next;
    }
    // A single grid has units of one size, so a launch takes ceil(units / warps) rounds of them:
    // its segment count is raised by up to a quarter where that fills the last round better
    // (the 4096^2 warped step: 147 x 128 units over 1824 warps fill their eleventh round to 32 %,
    // 147 x 124 units fill ten rounds to 99.9 %).
    int single_nty = 0;
    if (g->count == 1) {
        const GridDev &G = g->hg[0];
        const long long ntx = (G.ni + width - 1) / width;
        const int nty0 = (G.nj + ty - 1) / ty;
        double best = -1.0;
        for (int n = std::max(1, nty0 - nty0 / 8); n <= nty0 + nty0 / 4 && n <= G.nj; ++n) {
            const long long units = ntx * n;
            const long long rounds = (units + warps - 1) / warps;
            // useful fraction of the rounds, less the warm-up rows each extra segment re-reads
            const double eff = (double)units / (double)(rounds * warps) * (1.0 - (double)(H + 1) * n / (2.0 * G.nj));
            if (eff > best + 1e-9) { best = eff; single_nty = n; }
        }
    }
    // Rows next to an EXCHANGE side (H of them) read its ghost rows; they form segments of their
    // own, so that a slab can run its interior while its ghost rows are on their way
    // (roeam_rk_stage_part). Other grids are all interior.
    std::vector<int4> ug, edges_all;
    g->h_tile_base.assign(g->count + 1, 0);
    for (int k = 0; k < g->count; ++k) {
        GridDev &G = g->hg[k];
        const bool exS = G.bc[2] == ROEAM_BC_EXCHANGE, exN = G.bc[3] == ROEAM_BC_EXCHANGE;
        int lo = exS ? H : 0, hi = exN ? G.nj - H : G.nj;
        if (hi - lo < 1) lo = hi = 0;   // (a slab too thin for an interior: one edge segment)
        const int nin = hi - lo;
        G.ntx = (G.ni + width - 1) / width;
        int nseg = nin > 0 ? (single_nty > 0 ? single_nty : (nin + ty - 1) / ty) : 0;
        nseg = std::min(nseg, std::max(nin, 0));
        G.tile_base = (int)ug.size();
        g->h_tile_base[k] = G.tile_base;
        for (int sg = 0; sg < nseg; ++sg) {
            const int j0 = lo + (int)((long long)sg * nin / nseg), j1 = lo + (int)((long long)(sg + 1) * nin / nseg);
            for (int st = 0; st < G.ntx; ++st) ug.push_back(make_int4(k, st * width - H, j0, j1));
        }
        std::vector<std::pair<int, int>> eseg;
        if (nin == 0) eseg.emplace_back(0, G.nj);
        else {
            if (lo > 0) eseg.emplace_back(0, lo);
            if (hi < G.nj) eseg.emplace_back(hi, G.nj);
        }
        for (const auto &e : eseg)
            for (int st = 0; st < G.ntx; ++st) {
                ug.push_back(make_int4(k, st * width - H, e.first, e.second));
                edges_all.push_back(ug.back());
            }
        G.nty = nseg + (int)eseg.size();
        G.ntiles = (int)ug.size() - G.tile_base;
    }
    const int base = (int)ug.size();
    g->h_tile_base[g->count] = base;
    g->total_tiles = base;
    auto taller = [](const int4 &a, const int4 &b) { return (a.w - a.z) > (b.w - b.z); };
    std::vector<int4> ua(ug);
    std::stable_sort(ua.begin(), ua.end(), taller);
    // interior units (every unit that is not an edge unit) by height, then the edge units
    std::vector<int4> up;
    {
        std::vector<int4> interior;
        size_t e = 0;
        for (int k = 0; k < g->count; ++k)
            for (int t = g->h_tile_base[k]; t < g->h_tile_base[k + 1]; ++t) {
                const int4 q = ug[t];
                if (e < edges_all.size() && q.x == edges_all[e].x && q.y == edges_all[e].y && q.z == edges_all[e].z &&
                    q.w == edges_all[e].w) ++e;
                else interior.push_back(q);
            }
        std::stable_sort(interior.begin(), interior.end(), taller);
        up = interior;
        g->part_split = (int)up.size();
        up.insert(up.end(), edges_all.begin(), edges_all.end());
    }
    if (base > g->units_cap) {
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        cudaFree(g->d_units_grid);
        cudaFree(g->d_units_all);
        cudaFree(g->d_units_part);
        g->d_units_grid = g->d_units_all = g->d_units_part = nullptr;
        CUDA_TRY(cudaMalloc(&g->d_units_grid, sizeof(int4) * base));
        CUDA_TRY(cudaMalloc(&g->d_units_all, sizeof(int4) * base));
        CUDA_TRY(cudaMalloc(&g->d_units_part, sizeof(int4) * base));
        g->units_cap = base;
    }
    CUDA_TRY(cudaMemcpyAsync(g->d_grids, g->hg.data(), sizeof(GridDev) * g->count, cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaMemcpyAsync(g->d_units_grid, ug.data(), sizeof(int4) * base, cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaMemcpyAsync(g->d_units_all, ua.data(), sizeof(int4) * base, cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaMemcpyAsync(g->d_units_part, up.data(), sizeof(int4) * base, cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->nblocks = std::max(1, occ * g->num_sms);
    g->eff_ty = ty;
    g->eff_dyn = tc.dyn && stage_dynamic(g->muscl, g->curv);
    for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
    g->graphs.clear();
    return ROEAM_OK;
}

// roeam_step_host's unit table: the units of every chunk of grids, cut with the current tile
// shape's segment height halved (down to MIN_SEGMENT_ROWS) until the chunk alone has a unit for every
// resident warp, ordered by decreasing height within the chunk.
roeam_status setup_pipe_units(roeam_grid *g, const std::vector<std::pair<int, int>> &chunks)
{
    const int H = g->muscl ? 2 : 1;
    const int width = 32 - 2 * H;
    const long long warps = g->nblocks;
    std::vector<int4> up;
    std::vector<int> base;
    for (const auto &ch : chunks) {
        base.push_back((int)up.size());
        int ty = TILE_CFGS[g->tile_cfg].ty;
        for (;;) {
            long long units = 0;
            for (int k = ch.first; k < ch.second; ++k)
                units += (long long)((g->hg[k].ni + width - 1) / width) * ((g->hg[k].nj + ty - 1) / ty);
            if (units >= warps || ty <= MIN_SEGMENT_ROWS) break;
            const int next = std::max(MIN_SEGMENT_ROWS, ty / 2);
            if (next < 4) {
                // (below 4 rows only while the chunk's units still fit one round, as above)
                long long fit = 0;
                for (int k = ch.first; k < ch.second; ++k)
                    fit += (long long)((g->hg[k].ni + width - 1) / width) * ((g->hg[k].nj + next - 1) / next);
                if (fit > warps) break;
            }
            ty = next;
        }
        const size_t b0 = up.size();
        for (int k = ch.first; k < ch.second; ++k) {
            const GridDev &G = g->hg[k];
            const int nty = (G.nj + ty - 1) / ty, ntx = (G.ni + width - 1) / width;
            for (int sg = 0; sg < nty; ++sg) {
                const int j0 = (int)((long long)sg * G.nj / nty), j1 = (int)((long long)(sg + 1) * G.nj / nty);
                for (int st = 0; st < ntx; ++st) up.push_back(make_int4(k, st * width - H, j0, j1));
            }
        }
        std::stable_sort(up.begin() + b0, up.end(), [](const int4 &a, const int4 &b) { return (a.w - a.z) > (b.w - b.z); });
    }
    base.push_back((int)up.size());
    if ((int)up.size() > g->pipe_units_cap) {
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        cudaFree(g->d_units_pipe);
        g->d_units_pipe = nullptr;
        CUDA_TRY(cudaMalloc(&g->d_units_pipe, sizeof(int4) * up.size()));
        g->pipe_units_cap = (int)up.size();
    }
    CUDA_TRY(cudaMemcpy(g->d_units_pipe, up.data(), sizeof(int4) * up.size(), cudaMemcpyHostToDevice));
    g->pipe_chunks = chunks;
    g->pipe_tile_base = base;
    g->pipe_cfg = g->tile_cfg;
    return ROEAM_OK;
}

// The autotuner's workload key: the device and kernel family, and every grid's sizes,
// boundary kinds and scheme switches (FNV-1a over them); the time-step parameters do not
// change which shape is fastest.
std::string tune_key(const roeam_grid *g, double, int)
{
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](long long v) {
        for (int b = 0; b < 8; ++b) { h ^= (unsigned long long)((v >> (8 * b)) & 0xff); h *= 1099511628211ull; }
    };
    for (const GridDev &G : g->hg) {
        mix(G.ni); mix(G.nj); mix(G.soff >= 0);
        for (int s = 0; s < 4; ++s) mix(G.bc[s]);
        mix(G.limiter); mix(G.eps1); mix(G.use_s1); mix(G.xi_form); mix(G.scheme); mix(G.dup_mode); mix(G.ufix);
        mix(G.xi_roe);
    }
    char buf[160];
    std::snprintf(buf, sizeof(buf), "dev%d/sm%d/p%d/m%d/c%d/k%d/n%d/%016llx", g->device, g->num_sms, g->precision,
                  g->muscl, g->curv, g->kind, g->count, h);
    return std::string(buf);
}

template <typename T>
roeam_status upload_geometry(roeam_grid *g, const roeam_grid_desc *d)
{
    if (!g->curv) return ROEAM_OK;
    std::vector<T> hx(g->total_vert, T(0)), hy(g->total_vert, T(0));
    for (int k = 0; k < g->count; ++k) {
        const GridDev &G = g->hg[k];
        for (int J = 0; J <= G.nj; ++J)
            for (int I = 0; I <= G.ni; ++I) {
                const size_t s = (size_t)J * (G.ni + 1) + I;
                const size_t t = (size_t)G.voff + (size_t)J * G.vpitch + I;
                hx[t] = T(d[k].xv[s] - I * d[k].dx);
                hy[t] = T(d[k].yv[s] - J * d[k].dy);
            }
    }
    CUDA_TRY(cudaMemcpy(g->vdx, hx.data(), sizeof(T) * g->total_vert, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(g->vdy, hy.data(), sizeof(T) * g->total_vert, cudaMemcpyHostToDevice));
    return ROEAM_OK;
}

template <typename T>
roeam_status upload_coef(roeam_grid *g)
{
    std::vector<GridCoef<T>> h(g->count);
    for (int k = 0; k < g->count; ++k) {
        const GridDev &G = g->hg[k];
        GridCoef<T> &c = h[k];
        c.g = T(G.gamma);
        c.gm1 = T(G.gamma - 1.0);
        c.gm1i = T(1.0 / (G.gamma - 1.0));
        c.hgm1 = T(0.5 * (G.gamma - 1.0));
        // (the classical Roe flux does not use M_ref; its time-step rule is |U| + c: theta = 1)
        c.mr2 = T(G.scheme == ROEAM_SCHEME_ROE ? 1.0 : G.m_ref * G.m_ref);
        c.rr_thr = T(1e-5 * G.u_ref);
        c.eps2 = T(G.eps2);
        c.dx = T(G.dx);
        c.dy = T(G.dy);
        c.V = T(G.dx * G.dy);
        c.Vi = T(1.0 / (G.dx * G.dy));
        c.idx = T(1.0 / G.dx);
        c.idy = T(1.0 / G.dy);
        for (int s = 0; s < 4; ++s) c.inflow[s] = T(G.inflow[s]);
        c.harten = T(G.harten);
    }
    CUDA_TRY(cudaMalloc(&g->d_coef, sizeof(GridCoef<T>) * g->count));
    CUDA_TRY(cudaMemcpy(g->d_coef, h.data(), sizeof(GridCoef<T>) * g->count, cudaMemcpyHostToDevice));
    return ROEAM_OK;
}

// Stage-kernel arguments common to every mode.
template <typename T>
StageArgs<T> base_args(roeam_grid *g)
{
    StageArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.grids = g->d_grids;
    a.coef = (const GridCoef<T> *)g->d_coef;
    a.units = g->d_units_all;
    a.ngrids = g->count;
    a.tile_lo = 0;
    a.tile_hi = g->total_tiles;
    a.vdx = (const T *)g->vdx;
    a.vdy = (const T *)g->vdy;
    a.solid = g->solid;
    a.status = g->status;
    a.work = g->eff_dyn ? g->work : nullptr;
#ifdef ROEAM_DEBUG
    a.n_state = a.n_dst = g->total_elems;
    a.n_vert = g->total_vert;
    a.n_solid = g->total_solid;
#endif
    return a;
}

template <typename T>
roeam_status launch_step(roeam_grid *g, cudaStream_t s, long long step, double cfl, double dt_fixed)
{
    const int par = (int)(step & 1);
    unsigned long long *rd = g->rate + (size_t)par * g->count;
    unsigned long long *wr = g->rate + (size_t)(1 - par) * g->count;
    T *U = (T *)g->U, *A = (T *)g->A, *B = (T *)g->B;
    StageArgs<T> a = base_args<T>(g);
    a.mode = MODE_STAGE;
    a.rate_rd = rd;
    a.cfl = cfl;
    a.dt_fixed = dt_fixed;
    a.cfl_t = T(cfl);
    a.dt_fixed_t = T(dt_fixed);
    // Stage 1: U1 = U^n + dt R(U^n)
    a.src = U; a.un = U; a.dst = A; a.alpha = T(0); a.beta = T(1); a.rate_zero = wr; a.want_rate = 0;
    CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, s));
    // Stage 2: U2 = 3/4 U^n + 1/4 (U1 + dt R(U1))
    a.src = A; a.un = U; a.dst = B; a.alpha = T(0.75); a.beta = T(0.25); a.rate_zero = nullptr;
    CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, s));
    // Stage 3: U^{n+1} = 1/3 U^n + 2/3 (U2 + dt R(U2)), in place; rate of U^{n+1} for the next dt
    a.src = B; a.un = U; a.dst = U; a.alpha = T(1.0 / 3.0); a.beta = T(2.0 / 3.0); a.rate_wr = wr; a.want_rate = 1;
    CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, s));
    return ROEAM_OK;
}

// The rate output of a pack into the current step's rate slots (grids [lo, hi) of `slot`
// zeroed first on stream s), so that the next step takes its dt from the state just loaded.
template <typename T>
roeam_status rate_out(roeam_grid *g, int lo, int hi, cudaStream_t s, RateOut<T> &ro)
{
    unsigned long long *slot = g->rate + (size_t)(g->step & 1) * g->count;
    CUDA_TRY(cudaMemsetAsync(slot + lo, 0, sizeof(unsigned long long) * (hi - lo), s));
    ro.coef = (const GridCoef<T> *)g->d_coef;
    ro.vdx = (const T *)g->vdx;
    ro.vdy = (const T *)g->vdy;
    ro.solid = g->solid;
    ro.rate = slot;
    ro.curv = g->curv;
    return ROEAM_OK;
}

template <typename T>
roeam_status rk_steps(roeam_grid *g, double cfl, double dt_fixed, int nsteps)
{
    int left = nsteps;
    auto direct = [&]() -> roeam_status {
        roeam_status st = launch_step<T>(g, g->stream, g->step, cfl, dt_fixed);
        if (st != ROEAM_OK) return st;
        g->step += 1;
        g->launches += 3;
        left -= 1;
        return ROEAM_OK;
    };
    if (left > 0 && (g->step & 1)) {
        roeam_status st = direct();
        if (st != ROEAM_OK) return st;
    }
    if (left >= GRAPH_STEPS) {
        GraphKey key{cfl, dt_fixed};
        auto it = g->graphs.find(key);
        if (it == g->graphs.end() && g->graphs.size() >= MAX_GRAPHS) {
            // keep the cache small: a caller that varies dt_fixed call by call rebuilds graphs
            CUDA_TRY(cudaStreamSynchronize(g->stream));
            for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
            g->graphs.clear();
        }
        if (it == g->graphs.end()) {
            cudaGraph_t graph;
            CUDA_TRY(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
            for (int s = 0; s < GRAPH_STEPS; ++s) {
                roeam_status st = launch_step<T>(g, g->cap_stream, s, cfl, dt_fixed);
                if (st != ROEAM_OK) {
                    graph = nullptr;
                    cudaStreamEndCapture(g->cap_stream, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
            }
            CUDA_TRY(cudaStreamEndCapture(g->cap_stream, &graph));
            cudaGraphExec_t exec;
            cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            CUDA_TRY(e);
            it = g->graphs.emplace(key, exec).first;
        }
        while (left >= GRAPH_STEPS) {
            CUDA_TRY(cudaGraphLaunch(it->second, g->stream));
            g->step += GRAPH_STEPS;
            g->launches += 3 * GRAPH_STEPS;
            left -= GRAPH_STEPS;
        }
    }
    while (left > 0) {
        roeam_status st = direct();
        if (st != ROEAM_OK) return st;
    }
    return ROEAM_OK;
}

roeam_status read_status(roeam_grid *g)
{
    unsigned st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (st) {
        CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(unsigned), g->stream));
        if (st & ST_BOUNDS) return fail(ROEAM_E_BOUNDS, "a kernel index left its buffer (bounds-checked build)");
        if (st & ST_NONFINITE) return fail(ROEAM_E_NONFINITE, "non-finite state after a step");
        return fail(ROEAM_E_NONPOSITIVE, "non-positive density or pressure after a step");
    }
    return ROEAM_OK;
}

roeam_status check_idx(const roeam_grid *g, int idx)
{
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (idx < -1 || idx >= g->count) return fail(ROEAM_E_ARG, "grid_idx %d out of range [-1, %d)", idx, g->count);
    return ROEAM_OK;
}

// (H: the host arrays' element type, double or float; the staging buffer holds either)
template <typename T, typename H = double>
roeam_status do_set_state(roeam_grid *g, int idx, const H *cons)
{
    const int lo = idx < 0 ? 0 : idx, hi = idx < 0 ? g->count : idx + 1;
    const long long p0 = g->hg[lo].poff;
    const long long p1 = hi < g->count ? g->hg[hi].poff : g->total_packed;
    H *staging = (H *)g->staging;
    CUDA_TRY(cudaMemcpyAsync(staging + p0, cons, sizeof(H) * (p1 - p0), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaEventRecord(g->ev, g->stream));
    RateOut<T> ro;
    roeam_status st = rate_out<T>(g, lo, hi, g->stream, ro);
    if (st != ROEAM_OK) return st;
    CUDA_TRY(Launchers<T>::pack(g->d_grids, lo, hi, g->max_cells, (const H *)staging, (T *)g->U, g->stream, 0, &ro));
    g->launches += 1;
    CUDA_TRY(cudaEventSynchronize(g->ev));   // the caller's array may be reused once we return
    for (int k = lo; k < hi; ++k) g->state_set[k] = 1;
    return ROEAM_OK;
}

template <typename T, typename H = double>
roeam_status do_get(roeam_grid *g, int idx, const void *src, H *out)
{
    const int lo = idx < 0 ? 0 : idx, hi = idx < 0 ? g->count : idx + 1;
    const long long p0 = g->hg[lo].poff;
    const long long p1 = hi < g->count ? g->hg[hi].poff : g->total_packed;
    H *staging = (H *)g->staging;
    CUDA_TRY(Launchers<T>::unpack(g->d_grids, lo, hi, g->max_cells, (const T *)src, staging, g->stream));
    g->launches += 1;
    CUDA_TRY(cudaMemcpyAsync(out, staging + p0, sizeof(H) * (p1 - p0), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return ROEAM_OK;
}

// Device-pointer state I/O: the caller's float64 array lives on the handle's device. Work
// already submitted to the caller's stream `cs` is finished before the library reads or
// writes the array, and work submitted to `cs` afterwards waits for the library's kernels;
// the host does not wait. (cs equal to the handle's stream needs neither.)
roeam_status order_after(roeam_grid *g, cudaStream_t cs)
{
    if (cs == g->stream) return ROEAM_OK;
    CUDA_TRY(cudaEventRecord(g->ev_in, cs));
    CUDA_TRY(cudaStreamWaitEvent(g->stream, g->ev_in, 0));
    return ROEAM_OK;
}
roeam_status order_before(roeam_grid *g, cudaStream_t cs)
{
    if (cs == g->stream) return ROEAM_OK;
    CUDA_TRY(cudaEventRecord(g->ev_out, g->stream));
    CUDA_TRY(cudaStreamWaitEvent(cs, g->ev_out, 0));
    return ROEAM_OK;
}

template <typename T>
roeam_status do_set_state_device(roeam_grid *g, int idx, const double *cons, cudaStream_t cs)
{
    const int lo = idx < 0 ? 0 : idx, hi = idx < 0 ? g->count : idx + 1;
    roeam_status st = order_after(g, cs);
    if (st != ROEAM_OK) return st;
    RateOut<T> ro;
    st = rate_out<T>(g, lo, hi, g->stream, ro);
    if (st != ROEAM_OK) return st;
    CUDA_TRY(Launchers<T>::pack(g->d_grids, lo, hi, g->max_cells, cons, (T *)g->U, g->stream, g->hg[lo].poff, &ro));
    g->launches += 1;
    for (int k = lo; k < hi; ++k) g->state_set[k] = 1;
    return order_before(g, cs);
}

template <typename T>
roeam_status do_get_state_device(roeam_grid *g, int idx, double *out, cudaStream_t cs)
{
    const int lo = idx < 0 ? 0 : idx, hi = idx < 0 ? g->count : idx + 1;
    roeam_status st = order_after(g, cs);
    if (st != ROEAM_OK) return st;
    CUDA_TRY(Launchers<T>::unpack(g->d_grids, lo, hi, g->max_cells, (const T *)g->U, out, g->stream, 0,
                                  g->hg[lo].poff));
    g->launches += 1;
    return order_before(g, cs);
}

template <typename T>
roeam_status do_residual(roeam_grid *g, int idx, double *out)
{
    StageArgs<T> a = base_args<T>(g);
    a.mode = MODE_RESIDUAL;
    a.src = (const T *)g->U;
    a.un = (const T *)g->U;
    a.dst = (T *)g->A;
    if (idx >= 0) { a.units = g->d_units_grid; a.tile_lo = g->h_tile_base[idx]; a.tile_hi = g->h_tile_base[idx + 1]; }
    CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, g->stream));
    g->launches += 1;
    if (out) return do_get<T>(g, idx, g->A, out);
    return ROEAM_OK;
}

template <typename T>
roeam_status do_norm(roeam_grid *g, int idx, int kind, double out[4])
{
    StageArgs<T> a = base_args<T>(g);
    a.mode = MODE_NORM;
    a.work = nullptr;   // static units: each block's partials cover the same cells every call
    a.src = (const T *)g->U;
    a.un = (const T *)g->U;
    a.units = g->d_units_grid;
    a.tile_lo = g->h_tile_base[idx];
    a.tile_hi = g->h_tile_base[idx + 1];
    a.partials = g->partials;
    const int nb = std::min(g->nblocks, std::min(g->partial_rows, a.tile_hi - a.tile_lo));
    CUDA_TRY(cudaMemsetAsync(g->partials, 0, sizeof(double) * 8 * g->partial_rows, g->stream));
    CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, nb, g->stream));
    CUDA_TRY(launch_reduce_partials(g->partials, nb, 8, g->red_out, g->stream));
    g->launches += 2;
    CUDA_TRY(cudaMemcpyAsync(g->h_red, g->red_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    const double nf = g->hg[idx].nfluid > 0 ? g->hg[idx].nfluid : 1.0;
    for (int k = 0; k < 4; ++k) out[k] = kind == ROEAM_NORM_L2 ? std::sqrt(g->h_red[k] / nf) : g->h_red[4 + k];
    return ROEAM_OK;
}

template <typename T>
roeam_status do_totals(roeam_grid *g, int idx, double out[4])
{
    const long long n = (long long)g->hg[idx].ni * g->hg[idx].nj;
    const int nb = (int)std::min<long long>(std::min<long long>((n + 255) / 256, 2 * g->partial_rows), 1024);
    CUDA_TRY(Launchers<T>::totals(g->d_grids, (const GridCoef<T> *)g->d_coef, idx, (const T *)g->U,
                                  (const T *)g->vdx, (const T *)g->vdy, g->solid, g->partials, nb, g->curv, g->stream));
    CUDA_TRY(launch_reduce_partials(g->partials, nb, 4, g->red_out, g->stream));
    g->launches += 2;
    CUDA_TRY(cudaMemcpyAsync(g->h_red, g->red_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (int k = 0; k < 4; ++k) out[k] = g->h_red[k];
    return ROEAM_OK;
}

roeam_status validate(int count, const roeam_grid_desc *d)
{
    if (count < 1 || !d) return fail(ROEAM_E_ARG, "count must be >= 1 and descs non-null");
    if (count > 65535) return fail(ROEAM_E_ARG, "count must be <= 65535 grids per handle");
    for (int k = 0; k < count; ++k) {
        const roeam_grid_desc &q = d[k];
        const roeam_params &p = q.p;
        if (q.ni < 4 || q.nj < 4) return fail(ROEAM_E_ARG, "grid %d: ni, nj must be >= 4", k);
        if ((long long)q.ni * q.nj > (1ll << 28)) return fail(ROEAM_E_ARG, "grid %d: too many cells", k);
        if (!(p.gamma > 1.0)) return fail(ROEAM_E_ARG, "grid %d: gamma must be > 1", k);
        if (!(p.m_ref > 0.0)) return fail(ROEAM_E_ARG, "grid %d: m_ref must be > 0", k);
        if (!(p.u_ref > 0.0)) return fail(ROEAM_E_ARG, "grid %d: u_ref must be > 0", k);
        if (!(p.eps2 >= 0.0)) return fail(ROEAM_E_ARG, "grid %d: eps2 must be >= 0", k);
        if (p.eps1 != 0 && p.eps1 != 1) return fail(ROEAM_E_ARG, "grid %d: eps1 must be 0 or 1", k);
        if (p.use_s1 != 0 && p.use_s1 != 1) return fail(ROEAM_E_ARG, "grid %d: use_s1 must be 0 or 1", k);
        if (p.xi_form != 0 && p.xi_form != 1) return fail(ROEAM_E_ARG, "grid %d: xi_form must be 0 or 1", k);
        if (p.recon < 0 || p.recon > 2) return fail(ROEAM_E_ARG, "grid %d: recon must be 0, 1 or 2", k);
        if (p.scheme != ROEAM_SCHEME_ROEAM && p.scheme != ROEAM_SCHEME_ROE)
            return fail(ROEAM_E_ARG, "grid %d: scheme must be ROEAM_SCHEME_ROEAM or ROEAM_SCHEME_ROE", k);
        if (p.dup_mode < ROEAM_DUP_ROEAM || p.dup_mode > ROEAM_DUP_ROE)
            return fail(ROEAM_E_ARG, "grid %d: dup_mode must be 0, 1 or 2", k);
        if (p.no_ufix != 0 && p.no_ufix != 1) return fail(ROEAM_E_ARG, "grid %d: no_ufix must be 0 or 1", k);
        if (p.xi_roe != 0 && p.xi_roe != 1) return fail(ROEAM_E_ARG, "grid %d: xi_roe must be 0 or 1", k);
        if (p.reserved_ != 0) return fail(ROEAM_E_ARG, "grid %d: reserved_ must be 0", k);
        if (!(p.harten >= 0.0 && p.harten < 1.0)) return fail(ROEAM_E_ARG, "grid %d: harten must be in [0, 1)", k);
        if (p.scheme == ROEAM_SCHEME_ROE && (p.dup_mode || p.no_ufix || p.xi_roe))
            return fail(ROEAM_E_ARG, "grid %d: dup_mode, no_ufix and xi_roe are Roe-AM variants (scheme is ROE)", k);
        if (p.scheme == ROEAM_SCHEME_ROEAM && p.harten != 0.0)
            return fail(ROEAM_E_ARG, "grid %d: harten applies to the classical Roe scheme only", k);
        if (p.precision != 32 && p.precision != 64) return fail(ROEAM_E_ARG, "grid %d: precision must be 32 or 64", k);
        if (p.precision != d[0].p.precision) return fail(ROEAM_E_ARG, "grid %d: precision differs within the batch", k);
        if ((p.recon > 0) != (d[0].p.recon > 0))
            return fail(ROEAM_E_ARG, "grid %d: first-order and MUSCL grids cannot share a batch", k);
        if ((q.xv != nullptr) != (q.yv != nullptr)) return fail(ROEAM_E_ARG, "grid %d: give both xv and yv or neither", k);
        if ((q.xv != nullptr) != (d[0].xv != nullptr))
            return fail(ROEAM_E_ARG, "grid %d: Cartesian and curvilinear grids cannot share a batch", k);
        if (!q.xv && (!(q.dx > 0.0) || !(q.dy > 0.0))) return fail(ROEAM_E_ARG, "grid %d: dx, dy must be > 0", k);
        if (q.xv && (!(q.dx >= 0.0) || !(q.dy >= 0.0) || !std::isfinite(q.dx) || !std::isfinite(q.dy)))
            return fail(ROEAM_E_ARG, "grid %d: reference spacings dx, dy must be >= 0", k);
        if (q.xv) {
            // every cell must have positive area: vertices ordered so that i x j points out of the plane
            const int W = q.ni + 1;
            for (int J = 0; J < q.nj; ++J)
                for (int I = 0; I < q.ni; ++I) {
                    const size_t a = (size_t)J * W + I, b = a + W + 1, c = a + W, e = a + 1;
                    const double A = 0.5 * ((q.xv[b] - q.xv[a]) * (q.yv[c] - q.yv[e]) -
                                            (q.yv[b] - q.yv[a]) * (q.xv[c] - q.xv[e]));
                    if (!(A > 0.0))
                        return fail(ROEAM_E_ARG,
                                    "grid %d: cell (%d, %d) has area %g <= 0 (vertices must turn counter-clockwise "
                                    "from +i to +j)", k, I, J, A);
                }
        }
        for (int s = 0; s < 4; ++s)
            if (q.bc[s] < 0 || q.bc[s] > 4) return fail(ROEAM_E_ARG, "grid %d: bad boundary type on side %d", k, s);
        if (q.bc[0] == ROEAM_BC_EXCHANGE || q.bc[1] == ROEAM_BC_EXCHANGE)
            return fail(ROEAM_E_ARG, "grid %d: EXCHANGE is for the S and N sides (row slabs)", k);
        if ((q.bc[0] == ROEAM_BC_PERIODIC) != (q.bc[1] == ROEAM_BC_PERIODIC) ||
            (q.bc[2] == ROEAM_BC_PERIODIC) != (q.bc[3] == ROEAM_BC_PERIODIC))
            return fail(ROEAM_E_ARG, "grid %d: PERIODIC must be set on both sides of a direction", k);
        if (q.solid && (q.bc[0] == ROEAM_BC_PERIODIC || q.bc[2] == ROEAM_BC_PERIODIC))
            return fail(ROEAM_E_ARG, "grid %d: solid cells cannot be combined with periodic sides", k);
        for (int s = 0; s < 4; ++s)
            if (q.bc[s] == ROEAM_BC_INFLOW && !(q.inflow[0] > 0.0 && q.inflow[3] > 0.0))
                return fail(ROEAM_E_ARG, "grid %d: inflow density and pressure must be > 0", k);
    }
    return ROEAM_OK;
}

}  // namespace

namespace {

template <typename T>
roeam_status do_stage(roeam_grid *g, int stage, double dt, int part = 0)
{
    const int par = (int)(g->step & 1);
    unsigned long long *rd = g->rate + (size_t)par * g->count;
    unsigned long long *wr = g->rate + (size_t)(1 - par) * g->count;
    T *U = (T *)g->U, *A = (T *)g->A, *B = (T *)g->B;
    StageArgs<T> a = base_args<T>(g);
    a.mode = MODE_STAGE;
    a.rate_rd = rd;
    a.dt_fixed = dt;
    a.dt_fixed_t = T(dt);
    a.cfl_t = T(1);
    if (stage == 0) { a.src = U; a.un = U; a.dst = A; a.alpha = T(0); a.beta = T(1); a.rate_zero = wr; }
    else if (stage == 1) { a.src = A; a.un = U; a.dst = B; a.alpha = T(0.75); a.beta = T(0.25); }
    else { a.src = B; a.un = U; a.dst = U; a.alpha = T(1.0 / 3.0); a.beta = T(2.0 / 3.0); a.rate_wr = wr; a.want_rate = 1; }
    if (part != 0) {
        // interior units (part 1) or the units next to EXCHANGE sides (part 2); the next step's
        // rate slots are reset here rather than by a kernel, which either part may lack
        if (stage == 0 && part == 1) CUDA_TRY(cudaMemsetAsync(wr, 0, sizeof(unsigned long long) * g->count, g->stream));
        a.rate_zero = nullptr;
        a.units = g->d_units_part;
        a.tile_lo = part == 1 ? 0 : g->part_split;
        a.tile_hi = part == 1 ? g->part_split : g->total_tiles;
    }
    if (a.tile_hi > a.tile_lo) {
        CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, g->stream));
        g->launches += 1;
    }
    return ROEAM_OK;
}

// The state buffer that stage `stage` reads: U^n, U1 or U2.
void *stage_source(roeam_grid *g, int stage) { return stage == 0 ? g->U : (stage == 1 ? g->A : g->B); }

// Device address of the allocation-free residual's scratch array (defined at the end of this
// file); roeam_create_grid looks it up so that the array is committed on the device when a
// handle is made.
roeam_status noalloc_scratch(int device, void **out);

}  // namespace

namespace {

// One chunk of roeam_step_host, grids [lo, hi): the host-to-device copy of its packed input on
// the copy-in stream, the computation (the pack, which also takes the time-step rate, nsteps
// steps with the per-grid unit table, unpack) on the compute stream once the copy has landed, and the device-to-host copy on the
// copy-out stream once the computation is done. Chunks touch disjoint ranges of the staging
// buffer, the state planes, the rate slots and the host arrays, so the three streams never
// wait for one another except through the chunk's own two events.
template <typename T, typename H>
roeam_status pipe_chunk(roeam_grid *g, int chunk, int lo, int hi, int nsteps, double cfl, double dt_fixed,
                        const H *in, H *out, cudaEvent_t copied, cudaEvent_t computed)
{
    cudaStream_t s_in = g->pipe[0], s = g->pipe[1], s_out = g->pipe[2];
    const long long p0 = g->hg[lo].poff;
    const long long p1 = hi < g->count ? g->hg[hi].poff : g->total_packed;
    H *staging = (H *)g->staging;
    CUDA_TRY(cudaMemcpyAsync(staging + p0, in + p0, sizeof(H) * (p1 - p0), cudaMemcpyHostToDevice, s_in));
    CUDA_TRY(cudaEventRecord(copied, s_in));
    CUDA_TRY(cudaStreamWaitEvent(s, copied, 0));
    RateOut<T> ro;
    roeam_status st = rate_out<T>(g, lo, hi, s, ro);
    if (st != ROEAM_OK) return st;
    CUDA_TRY(Launchers<T>::pack(g->d_grids, lo, hi, g->max_cells, (const H *)staging, (T *)g->U, s, 0, &ro));
    T *U = (T *)g->U, *A = (T *)g->A, *B = (T *)g->B;
    StageArgs<T> a = base_args<T>(g);
    a.units = g->d_units_pipe;
    a.tile_lo = g->pipe_tile_base[chunk];
    a.tile_hi = g->pipe_tile_base[chunk + 1];
    a.mode = MODE_STAGE;
    a.cfl = cfl;
    a.dt_fixed = dt_fixed;
    a.cfl_t = T(cfl);
    a.dt_fixed_t = T(dt_fixed);
    for (long long st = g->step; st < g->step + nsteps; ++st) {
        const int par = (int)(st & 1);
        a.rate_rd = g->rate + (size_t)par * g->count;
        unsigned long long *wr = g->rate + (size_t)(1 - par) * g->count;
        CUDA_TRY(cudaMemsetAsync(wr + lo, 0, sizeof(unsigned long long) * (hi - lo), s));
        a.rate_zero = nullptr;
        a.src = U; a.un = U; a.dst = A; a.alpha = T(0); a.beta = T(1); a.want_rate = 0; a.rate_wr = nullptr;
        CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, s));
        a.src = A; a.dst = B; a.alpha = T(0.75); a.beta = T(0.25);
        CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, s));
        a.src = B; a.dst = U; a.alpha = T(1.0 / 3.0); a.beta = T(2.0 / 3.0); a.rate_wr = wr; a.want_rate = 1;
        CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, s));
    }
    CUDA_TRY(Launchers<T>::unpack(g->d_grids, lo, hi, g->max_cells, (const T *)g->U, staging, s));
    CUDA_TRY(cudaEventRecord(computed, s));
    CUDA_TRY(cudaStreamWaitEvent(s_out, computed, 0));
    CUDA_TRY(cudaMemcpyAsync(out + p0, staging + p0, sizeof(H) * (p1 - p0), cudaMemcpyDeviceToHost, s_out));
    g->launches += 2 + 3ull * nsteps;
    return ROEAM_OK;
}

}  // namespace

namespace roeam {
// Records a message for roeam_last_error() from the other host translation units.
int record_error(int status, const char *msg)
{
    g_last_error = msg;
    return status;
}
}  // namespace roeam

extern "C" {

const char *roeam_last_error(void) { return g_last_error.c_str(); }

int roeam_version(void) { return 10000; }

roeam_status roeam_create_grid(int count, const roeam_grid_desc *descs, int device, void *cuda_stream,
                               roeam_grid **out)
{
    if (!out) return fail(ROEAM_E_ARG, "out must be non-null");
    *out = nullptr;
    roeam_status st = validate(count, descs);
    if (st != ROEAM_OK) return st;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(ROEAM_E_ARG, "device %d not present (%d devices)", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    int num_sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));

    roeam_grid *g = new roeam_grid();
    g->device = device;
    g->stream = (cudaStream_t)cuda_stream;
    g->count = count;
    g->precision = descs[0].p.precision;
    g->esize = g->precision == 32 ? 4 : 8;
    g->muscl = descs[0].p.recon > 0;
    g->curv = descs[0].xv != nullptr;
    g->num_sms = num_sms;
    g->hg.resize(count);
    g->state_set.assign(count, 0);
    long long off = 0, voff = 0, soff = 0, poff = 0;
    bool any_solid = false;
    for (int k = 0; k < count; ++k) {
        const roeam_grid_desc &q = descs[k];
        GridDev &G = g->hg[k];
        std::memset(&G, 0, sizeof(G));
        G.ni = q.ni;
        G.nj = q.nj;
        G.pitch = (int)round_up(q.ni, 32);
        const bool exch = q.bc[2] == ROEAM_BC_EXCHANGE || q.bc[3] == ROEAM_BC_EXCHANGE;
        // (a grid with an EXCHANGE side keeps two ghost rows below and above in its planes)
        G.plane = (long long)(q.nj + (exch ? 4 : 0)) * G.pitch;
        G.off = off + (exch ? 2ll * G.pitch : 0);
        off += 4 * G.plane;
        if (g->curv) {
            // (an EXCHANGE grid also keeps two ghost vertex rows below and above, roeam_set_halo_vertices)
            G.vpitch = (int)round_up(q.ni + 1, 32);
            G.voff = voff + (exch ? 2ll * G.vpitch : 0);
            voff += (long long)(q.nj + 1 + (exch ? 4 : 0)) * G.vpitch;
        } else {
            G.voff = -1;
        }
        long long nf = (long long)q.ni * q.nj;
        if (q.solid) {
            // (an EXCHANGE grid also keeps two ghost mask rows below and above, roeam_set_halo_solid)
            G.soff = soff + (exch ? 2ll * q.ni : 0);
            soff += round_up((long long)q.ni * (q.nj + (exch ? 4 : 0)), 256);
            any_solid = true;
            for (long long c = 0; c < (long long)q.ni * q.nj; ++c) nf -= q.solid[c] ? 1 : 0;
        } else {
            G.soff = -1;
        }
        G.nfluid = (double)nf;
        G.poff = poff;
        poff += 4ll * q.ni * q.nj;
        g->max_cells = std::max(g->max_cells, q.ni * q.nj);
        for (int s = 0; s < 4; ++s) G.bc[s] = q.bc[s];
        bool walls = q.solid != nullptr;
        for (int s = 0; s < 4; ++s)
            if (q.bc[s] == ROEAM_BC_WALL) walls = true;
        const bool ablation = q.p.scheme != ROEAM_SCHEME_ROEAM || q.p.dup_mode != ROEAM_DUP_ROEAM || q.p.no_ufix ||
                              q.p.xi_roe;
        if (ablation) g->kind = KIND_ABLATION;
        else if (walls && g->kind == KIND_PLAIN) g->kind = KIND_WALLS;
        for (int s = 0; s < 4; ++s) G.inflow[s] = q.inflow[s];
        G.limiter = q.p.recon;
        G.eps1 = q.p.eps1;
        G.use_s1 = q.p.use_s1;
        G.xi_form = q.p.xi_form;
        G.scheme = q.p.scheme;
        G.dup_mode = q.p.dup_mode;
        G.ufix = q.p.no_ufix ? 0 : 1;
        G.xi_roe = q.p.xi_roe;
        G.harten = q.p.harten;
        G.gamma = q.p.gamma;
        G.m_ref = q.p.m_ref;
        G.u_ref = q.p.u_ref;
        G.eps2 = q.p.eps2;
        G.dx = q.dx;
        G.dy = q.dy;
    }
    g->total_elems = off;
    g->total_vert = voff;
    g->total_packed = poff;
    g->total_solid = soff;

    auto cleanup = [&](roeam_status s) { roeam_destroy_grid(g); return s; };
#define CREATE_TRY(expr)                                                                                        \
    do {                                                                                                        \
        cudaError_t e_ = (expr);                                                                                \
        if (e_ != cudaSuccess)                                                                                  \
            return cleanup(fail(e_ == cudaErrorMemoryAllocation ? ROEAM_E_OOM : ROEAM_E_CUDA, "%s: %s", #expr, \
                                cudaGetErrorString(e_)));                                                       \
    } while (0)

    CREATE_TRY(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    CREATE_TRY(cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming));
    CREATE_TRY(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
    CREATE_TRY(cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming));
    CREATE_TRY(cudaMalloc(&g->d_grids, sizeof(GridDev) * count));
    const size_t sbytes = g->esize * (size_t)g->total_elems;
    CREATE_TRY(cudaMalloc(&g->U, sbytes));
    CREATE_TRY(cudaMalloc(&g->A, sbytes));
    CREATE_TRY(cudaMalloc(&g->B, sbytes));
#ifdef ROEAM_DEBUG
    // bounds-checked builds fill the state buffers with NaN (padding columns, ghost rows not yet
    // set): a read of them that reached a written cell would show as a non-finite state
    const int fill = 0xFF;
#else
    const int fill = 0;
#endif
    CREATE_TRY(cudaMemset(g->U, fill, sbytes));
    CREATE_TRY(cudaMemset(g->A, fill, sbytes));
    CREATE_TRY(cudaMemset(g->B, fill, sbytes));
    if (g->curv) {
        CREATE_TRY(cudaMalloc(&g->vdx, g->esize * (size_t)g->total_vert));
        CREATE_TRY(cudaMalloc(&g->vdy, g->esize * (size_t)g->total_vert));
    }
    if (any_solid) {
        CREATE_TRY(cudaMalloc(&g->solid, (size_t)g->total_solid));
        std::vector<uint8_t> hs(g->total_solid, 0);
        for (int k = 0; k < count; ++k)
            if (descs[k].solid)
                for (long long c = 0; c < (long long)descs[k].ni * descs[k].nj; ++c)
                    hs[g->hg[k].soff + c] = descs[k].solid[c] ? 1 : 0;
        CREATE_TRY(cudaMemcpy(g->solid, hs.data(), hs.size(), cudaMemcpyHostToDevice));
    }
    CREATE_TRY(cudaMalloc(&g->staging, sizeof(double) * (size_t)g->total_packed));
    CREATE_TRY(cudaMalloc(&g->rate, sizeof(unsigned long long) * 2 * count));
    CREATE_TRY(cudaMemset(g->rate, 0, sizeof(unsigned long long) * 2 * count));
    CREATE_TRY(cudaMalloc(&g->status, sizeof(unsigned)));
    CREATE_TRY(cudaMemset(g->status, 0, sizeof(unsigned)));
    CREATE_TRY(cudaMalloc(&g->work, 2 * sizeof(unsigned)));
    CREATE_TRY(cudaMemset(g->work, 0, 2 * sizeof(unsigned)));
    g->partial_rows = 4 * 1024;
    CREATE_TRY(cudaMalloc(&g->partials, sizeof(double) * 8 * g->partial_rows));
    CREATE_TRY(cudaMalloc(&g->red_out, sizeof(double) * 8));
    CREATE_TRY(cudaMallocHost(&g->h_red, sizeof(double) * 8));
    CREATE_TRY(cudaMallocHost(&g->h_rate, sizeof(unsigned long long) * count));
    st = g->precision == 32 ? upload_geometry<float>(g, descs) : upload_geometry<double>(g, descs);
    if (st != ROEAM_OK) return cleanup(st);
    st = g->precision == 32 ? upload_coef<float>(g) : upload_coef<double>(g);
    if (st != ROEAM_OK) return cleanup(st);
    st = setup_tiles(g, 0);
    if (st != ROEAM_OK) return cleanup(st);
    // Load the module that holds the allocation-free residual's scratch array now (CUDA loads
    // modules lazily, and committing the array is an allocation), so that a caller which makes
    // its handles at start-up has the array before it stops allocating.
    void *scratch = nullptr;
    st = noalloc_scratch(device, &scratch);
    if (st != ROEAM_OK) return cleanup(st);
#undef CREATE_TRY
    *out = g;
    return ROEAM_OK;
}

void roeam_destroy_grid(roeam_grid *g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream); else cudaDeviceSynchronize();
    for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(g->d_grids);
    cudaFree(g->d_coef);
    cudaFree(g->d_units_grid);
    cudaFree(g->d_units_all);
    cudaFree(g->d_units_part);
    cudaFree(g->d_units_pipe);
    cudaFree(g->U);
    cudaFree(g->A);
    cudaFree(g->B);
    cudaFree(g->vdx);
    cudaFree(g->vdy);
    cudaFree(g->solid);
    cudaFree(g->staging);
    cudaFree(g->rate);
    cudaFree(g->status);
    cudaFree(g->work);
    cudaFree(g->partials);
    cudaFree(g->red_out);
    if (g->h_red) cudaFreeHost(g->h_red);
    if (g->h_rate) cudaFreeHost(g->h_rate);
    if (g->ev) cudaEventDestroy(g->ev);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    for (int k = 0; k < 3; ++k)
        if (g->pipe[k]) cudaStreamDestroy(g->pipe[k]);
    for (cudaEvent_t e : g->pipe_ev) cudaEventDestroy(e);
    delete g;
}

roeam_status roeam_set_state(roeam_grid *g, int grid_idx, const double *cons)
{
    const Range range_("roeam_set_state");
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (!cons) return fail(ROEAM_E_ARG, "cons must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    return g->precision == 32 ? do_set_state<float>(g, grid_idx, cons) : do_set_state<double>(g, grid_idx, cons);
}

// A device pointer of the handle's device (or managed memory), else ROEAM_E_ARG.
static roeam_status check_device_ptr(const roeam_grid *g, const void *p, const char *what)
{
    if (!p) return fail(ROEAM_E_ARG, "%s must be non-null", what);
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(ROEAM_E_ARG, "%s is not a CUDA pointer", what);
    }
    if (at.type == cudaMemoryTypeManaged) return ROEAM_OK;
    if (at.type != cudaMemoryTypeDevice || at.device != g->device)
        return fail(ROEAM_E_ARG, "%s must be device memory of device %d", what, g->device);
    if (((uintptr_t)p & 7) != 0) return fail(ROEAM_E_ARG, "%s must be 8-byte aligned", what);
    return ROEAM_OK;
}

roeam_status roeam_set_state_device(roeam_grid *g, int grid_idx, const double *cons_dev, void *cuda_stream)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    CUDA_TRY(cudaSetDevice(g->device));
    st = check_device_ptr(g, cons_dev, "cons_dev");
    if (st != ROEAM_OK) return st;
    const cudaStream_t cs = (cudaStream_t)cuda_stream;
    return g->precision == 32 ? do_set_state_device<float>(g, grid_idx, cons_dev, cs)
                              : do_set_state_device<double>(g, grid_idx, cons_dev, cs);
}

roeam_status roeam_get_state_device(roeam_grid *g, int grid_idx, double *cons_out_dev, void *cuda_stream)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    CUDA_TRY(cudaSetDevice(g->device));
    st = check_device_ptr(g, cons_out_dev, "cons_out_dev");
    if (st != ROEAM_OK) return st;
    const cudaStream_t cs = (cudaStream_t)cuda_stream;
    return g->precision == 32 ? do_get_state_device<float>(g, grid_idx, cons_out_dev, cs)
                              : do_get_state_device<double>(g, grid_idx, cons_out_dev, cs);
}

roeam_status roeam_get_state(roeam_grid *g, int grid_idx, double *cons_out)
{
    const Range range_("roeam_get_state");
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (!cons_out) return fail(ROEAM_E_ARG, "cons_out must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    st = g->precision == 32 ? do_get<float>(g, grid_idx, g->U, cons_out) : do_get<double>(g, grid_idx, g->U, cons_out);
    if (st != ROEAM_OK) return st;
    return read_status(g);
}

roeam_status roeam_flux_residual(roeam_grid *g, int grid_idx, double *res_out)
{
    const Range range_("roeam_flux_residual");
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    for (int k = 0; k < g->count; ++k)
        if ((grid_idx < 0 || grid_idx == k) && !g->state_set[k]) return fail(ROEAM_E_STATE, "state of grid %d not set", k);
    CUDA_TRY(cudaSetDevice(g->device));
    return g->precision == 32 ? do_residual<float>(g, grid_idx, res_out) : do_residual<double>(g, grid_idx, res_out);
}

roeam_status roeam_rk_step(roeam_grid *g, double cfl, double dt_fixed, int nsteps, double *dt_last)
{
    const Range range_("roeam_rk_step");
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (nsteps < 0) return fail(ROEAM_E_ARG, "nsteps must be >= 0");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(ROEAM_E_ARG, "need cfl > 0 or dt_fixed > 0");
    if (!std::isfinite(cfl) || !std::isfinite(dt_fixed)) return fail(ROEAM_E_ARG, "cfl and dt_fixed must be finite");
    for (int k = 0; k < g->count; ++k)
        if (!g->state_set[k]) return fail(ROEAM_E_STATE, "state of grid %d not set", k);
    if (g->stage_next != 0 || g->part_next != 0) return fail(ROEAM_E_STATE, "a step run by roeam_rk_stage is unfinished");
    CUDA_TRY(cudaSetDevice(g->device));
    const long long step0 = g->step;
    roeam_status st = g->precision == 32 ? rk_steps<float>(g, cfl, dt_fixed, nsteps)
                                         : rk_steps<double>(g, cfl, dt_fixed, nsteps);
    if (st != ROEAM_OK) return st;
    if (dt_last) {
        if (nsteps == 0 || dt_fixed > 0.0) {
            for (int k = 0; k < g->count; ++k) dt_last[k] = nsteps == 0 ? 0.0 : dt_fixed;
        } else {
            const int par = (int)((step0 + nsteps - 1) & 1);   // slot the last step read its rate from
            CUDA_TRY(cudaMemcpyAsync(g->h_rate, g->rate + (size_t)par * g->count,
                                     sizeof(unsigned long long) * g->count, cudaMemcpyDeviceToHost, g->stream));
            CUDA_TRY(cudaStreamSynchronize(g->stream));
            for (int k = 0; k < g->count; ++k) {
                double r;
                if (g->precision == 32) {
                    float f;
                    const uint32_t lo = (uint32_t)(g->h_rate[k] & 0xffffffffull);
                    std::memcpy(&f, &lo, sizeof(float));
                    dt_last[k] = (double)(float(cfl) / f);
                } else {
                    std::memcpy(&r, g->h_rate + k, sizeof(double));
                    dt_last[k] = cfl / r;
                }
            }
        }
        return read_status(g);
    }
    return ROEAM_OK;
}

roeam_status roeam_residual_norm(roeam_grid *g, int grid_idx, int kind, double out[4])
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (grid_idx < 0) return fail(ROEAM_E_ARG, "residual_norm needs one grid (grid_idx >= 0)");
    if (kind != ROEAM_NORM_L2 && kind != ROEAM_NORM_LINF) return fail(ROEAM_E_ARG, "bad norm kind %d", kind);
    if (!out) return fail(ROEAM_E_ARG, "out must be non-null");
    if (!g->state_set[grid_idx]) return fail(ROEAM_E_STATE, "state of grid %d not set", grid_idx);
    CUDA_TRY(cudaSetDevice(g->device));
    st = g->precision == 32 ? do_norm<float>(g, grid_idx, kind, out) : do_norm<double>(g, grid_idx, kind, out);
    if (st != ROEAM_OK) return st;
    return read_status(g);
}

roeam_status roeam_conserved_totals(roeam_grid *g, int grid_idx, double out[4])
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (grid_idx < 0) return fail(ROEAM_E_ARG, "conserved_totals needs one grid (grid_idx >= 0)");
    if (!out) return fail(ROEAM_E_ARG, "out must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    st = g->precision == 32 ? do_totals<float>(g, grid_idx, out) : do_totals<double>(g, grid_idx, out);
    if (st != ROEAM_OK) return st;
    return read_status(g);
}

roeam_status roeam_check(roeam_grid *g)
{
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    CUDA_TRY(cudaSetDevice(g->device));
    return read_status(g);
}

int roeam_tile_config_count(void) { return NUM_TILE_CFGS; }

roeam_status roeam_tile_config_info(int cfg, int *tx, int *ty, int *threads)
{
    if (cfg < 0 || cfg >= NUM_TILE_CFGS) return fail(ROEAM_E_ARG, "tile config %d out of range", cfg);
    if (tx) *tx = TILE_CFGS[cfg].tx;
    if (ty) *ty = TILE_CFGS[cfg].ty;
    if (threads) *threads = TILE_CFGS[cfg].nt;
    return ROEAM_OK;
}

roeam_status roeam_set_tile_config(roeam_grid *g, int cfg)
{
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (cfg < 0 || cfg >= NUM_TILE_CFGS) return fail(ROEAM_E_ARG, "tile config %d out of range", cfg);
    if (g->part_next != 0) return fail(ROEAM_E_STATE, "the edge part of a stage is due");
    CUDA_TRY(cudaSetDevice(g->device));
    return setup_tiles(g, cfg);
}

roeam_status roeam_autotune(roeam_grid *g, double cfl, int steps, int *best_cfg, double *ms_per_step)
{
    const Range range_("roeam_autotune");
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (steps < 1 || !(cfl > 0.0)) return fail(ROEAM_E_ARG, "need steps >= 1 and cfl > 0");
    if (g->stage_next != 0 || g->part_next != 0) return fail(ROEAM_E_STATE, "a step run by roeam_rk_stage is unfinished");
    for (int k = 0; k < g->count; ++k)
        if (!g->state_set[k]) return fail(ROEAM_E_STATE, "state of grid %d not set", k);
    CUDA_TRY(cudaSetDevice(g->device));
    const size_t sbytes = g->esize * (size_t)g->total_elems;
    const size_t rbytes = sizeof(unsigned long long) * 2 * g->count;
    void *save = nullptr;
    CUDA_TRY(cudaMalloc(&save, sbytes + rbytes));
    const long long step0 = g->step;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    roeam_status st = ROEAM_OK;
    int best = g->tile_cfg;
    double best_ms = 1e300;
    double times[NUM_TILE_CFGS];
    const std::string key = tune_key(g, cfl, steps);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            // this workload was tuned before in this process: take its result without timing
            cudaFree(save);
            st = setup_tiles(g, it->second.best);
            if (st != ROEAM_OK) return st;
            if (best_cfg) *best_cfg = it->second.best;
            if (ms_per_step)
                for (int c = 0; c < NUM_TILE_CFGS; ++c) ms_per_step[c] = it->second.ms[c];
            return ROEAM_OK;
        }
    }
    auto run = [&]() -> roeam_status {
        if (cudaMemcpyAsync(save, g->U, sbytes, cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess ||
            cudaMemcpyAsync((char *)save + sbytes, g->rate, rbytes, cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            return fail(ROEAM_E_CUDA, "autotune setup failed");
        std::vector<std::pair<int, int>> seen;   // (segment height, schedule) already timed, and by which shape
        for (int cfg = 0; cfg < NUM_TILE_CFGS; ++cfg) {
            roeam_status s2 = setup_tiles(g, cfg);
            if (s2 != ROEAM_OK) return s2;
            // shapes that give the same units and schedule (small batches halve every height to the
            // same one; kernels without dynamic scheduling) are timed once
            int same = -1;
            for (size_t q = 0; q < seen.size(); ++q)
                if (seen[q].first == g->eff_ty * 2 + g->eff_dyn) same = seen[q].second;
            if (same >= 0) {
                times[cfg] = times[same];
                continue;
            }
            seen.emplace_back(g->eff_ty * 2 + g->eff_dyn, cfg);
            double per = 1e300;
            for (int rep = 0; rep < 2; ++rep) {   // best of two timings
                s2 = g->precision == 32 ? rk_steps<float>(g, cfl, 0.0, 1) : rk_steps<double>(g, cfl, 0.0, 1);   // warm-up
                if (s2 != ROEAM_OK) return s2;
                CUDA_TRY(cudaEventRecord(e0, g->stream));
                s2 = g->precision == 32 ? rk_steps<float>(g, cfl, 0.0, steps) : rk_steps<double>(g, cfl, 0.0, steps);
                if (s2 != ROEAM_OK) return s2;
                CUDA_TRY(cudaEventRecord(e1, g->stream));
                CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                per = std::min(per, (double)ms / steps);
                // restore the state, the rate slots and the step parity
                CUDA_TRY(cudaMemcpyAsync(g->U, save, sbytes, cudaMemcpyDeviceToDevice, g->stream));
                CUDA_TRY(cudaMemcpyAsync(g->rate, (char *)save + sbytes, rbytes, cudaMemcpyDeviceToDevice, g->stream));
                g->step = step0;
            }
            times[cfg] = per;
            if (per < best_ms) { best_ms = per; best = cfg; }
        }
        return setup_tiles(g, best);
    };
    st = run();
    cudaStreamSynchronize(g->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (st != ROEAM_OK) return st;
    if (best_cfg) *best_cfg = best;
    if (ms_per_step)
        for (int c = 0; c < NUM_TILE_CFGS; ++c) ms_per_step[c] = times[c];
    st = read_status(g);
    if (st == ROEAM_OK) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        TuneResult r;
        r.best = best;
        for (int c = 0; c < NUM_TILE_CFGS; ++c) r.ms[c] = times[c];
        g_tune_cache[key] = r;
    }
    return st;
}

unsigned long long roeam_launch_count(const roeam_grid *g) { return g ? g->launches : 0ull; }

long long roeam_cell_count(const roeam_grid *g, int grid_idx)
{
    if (!g || grid_idx < -1 || grid_idx >= g->count) return -1;
    if (grid_idx >= 0) return (long long)g->hg[grid_idx].ni * g->hg[grid_idx].nj;
    return g->total_packed / 4;
}


// ---- stage-by-stage stepping and ghost rows (row slabs of one grid on several GPUs)

roeam_status roeam_max_rate(roeam_grid *g, double *rate_out)
{
    if (!g || !rate_out) return fail(ROEAM_E_ARG, "null argument");
    CUDA_TRY(cudaSetDevice(g->device));
    const int par = (int)(g->step & 1);
    CUDA_TRY(cudaMemcpyAsync(g->h_rate, g->rate + (size_t)par * g->count, sizeof(unsigned long long) * g->count,
                             cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (int k = 0; k < g->count; ++k) {
        if (g->precision == 32) {
            float f;
            const uint32_t lo = (uint32_t)(g->h_rate[k] & 0xffffffffull);
            std::memcpy(&f, &lo, sizeof(float));
            rate_out[k] = (double)f;
        } else {
            std::memcpy(&rate_out[k], g->h_rate + k, sizeof(double));
        }
    }
    return read_status(g);
}


roeam_status roeam_rk_stage(roeam_grid *g, int stage, double dt)
{
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (stage < 0 || stage > 2) return fail(ROEAM_E_ARG, "stage must be 0, 1 or 2");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ROEAM_E_ARG, "dt must be finite and > 0");
    return roeam_rk_stage_part(g, stage, dt, ROEAM_PART_ALL);
}

roeam_status roeam_rk_stage_part(roeam_grid *g, int stage, double dt, int part)
{
    const Range range_("roeam_rk_stage_part");
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (stage < 0 || stage > 2) return fail(ROEAM_E_ARG, "stage must be 0, 1 or 2");
    if (part < ROEAM_PART_ALL || part > ROEAM_PART_EDGES) return fail(ROEAM_E_ARG, "part must be 0, 1 or 2");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ROEAM_E_ARG, "dt must be finite and > 0");
    if (stage != g->stage_next) return fail(ROEAM_E_STATE, "stage %d expected, %d given", g->stage_next, stage);
    if (g->part_next == 1 && part != ROEAM_PART_EDGES)
        return fail(ROEAM_E_STATE, "the edge part of stage %d is due", stage);
    if (g->part_next == 0 && part == ROEAM_PART_EDGES)
        return fail(ROEAM_E_STATE, "the interior part of stage %d comes first", stage);
    for (int k = 0; k < g->count; ++k)
        if (!g->state_set[k]) return fail(ROEAM_E_STATE, "state of grid %d not set", k);
    CUDA_TRY(cudaSetDevice(g->device));
    roeam_status st = g->precision == 32 ? do_stage<float>(g, stage, dt, part) : do_stage<double>(g, stage, dt, part);
    if (st != ROEAM_OK) return st;
    if (part == ROEAM_PART_INTERIOR) {
        g->part_next = 1;
        return ROEAM_OK;
    }
    g->part_next = 0;
    g->stage_next = (stage + 1) % 3;
    if (stage == 2) g->step += 1;
    return ROEAM_OK;
}

roeam_status roeam_edge_rows(roeam_grid *g, int grid_idx, int side, int stage, void *dst)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (grid_idx < 0) return fail(ROEAM_E_ARG, "edge rows need one grid (grid_idx >= 0)");
    if (side != 2 && side != 3) return fail(ROEAM_E_ARG, "side must be 2 (S) or 3 (N)");
    if (stage < 0 || stage > 2) return fail(ROEAM_E_ARG, "stage must be 0, 1 or 2");
    if (!dst) return fail(ROEAM_E_ARG, "dst must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    const GridDev &G = g->hg[grid_idx];
    const int r0 = side == 2 ? 0 : G.nj - 2;
    const char *base = (const char *)stage_source(g, stage) + g->esize * (size_t)G.off;
    for (int k = 0; k < 4; ++k)
        CUDA_TRY(cudaMemcpy2DAsync((char *)dst + g->esize * (size_t)(2 * k * G.ni), g->esize * G.ni,
                                   base + g->esize * (size_t)(k * G.plane + (long long)r0 * G.pitch),
                                   g->esize * G.pitch, g->esize * G.ni, 2, cudaMemcpyDefault, g->stream));
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, dst) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
    return ROEAM_OK;
}

roeam_status roeam_set_halo(roeam_grid *g, int grid_idx, int side, int stage, const void *src)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (grid_idx < 0) return fail(ROEAM_E_ARG, "ghost rows need one grid (grid_idx >= 0)");
    if (side != 2 && side != 3) return fail(ROEAM_E_ARG, "side must be 2 (S) or 3 (N)");
    const GridDev &G = g->hg[grid_idx];
    if (G.bc[side] != ROEAM_BC_EXCHANGE) return fail(ROEAM_E_ARG, "side %d of grid %d is not EXCHANGE", side, grid_idx);
    if (stage < 0 || stage > 2) return fail(ROEAM_E_ARG, "stage must be 0, 1 or 2");
    if (!src) return fail(ROEAM_E_ARG, "src must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    const long long r0 = side == 2 ? -2 : G.nj;
    char *base = (char *)stage_source(g, stage) + g->esize * (size_t)(G.off + r0 * G.pitch);
    for (int k = 0; k < 4; ++k)
        CUDA_TRY(cudaMemcpy2DAsync(base + g->esize * (size_t)(k * G.plane), g->esize * G.pitch,
                                   (const char *)src + g->esize * (size_t)(2 * k * G.ni), g->esize * G.ni,
                                   g->esize * G.ni, 2, cudaMemcpyDefault, g->stream));
    // a host source (page-locked memory copies asynchronously) may be reused once this returns
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, src) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        CUDA_TRY(cudaStreamSynchronize(g->stream));
    }
    return ROEAM_OK;
}

roeam_status roeam_set_halo_solid(roeam_grid *g, int grid_idx, int side, const uint8_t *rows)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (grid_idx < 0) return fail(ROEAM_E_ARG, "ghost rows need one grid (grid_idx >= 0)");
    if (side != 2 && side != 3) return fail(ROEAM_E_ARG, "side must be 2 (S) or 3 (N)");
    const GridDev &G = g->hg[grid_idx];
    if (G.bc[side] != ROEAM_BC_EXCHANGE) return fail(ROEAM_E_ARG, "side %d of grid %d is not EXCHANGE", side, grid_idx);
    if (G.soff < 0) return fail(ROEAM_E_ARG, "grid %d has no solid mask (give it one, all zeros if need be)", grid_idx);
    if (!rows) return fail(ROEAM_E_ARG, "rows must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    std::vector<uint8_t> h(2 * (size_t)G.ni);
    for (size_t c = 0; c < h.size(); ++c) h[c] = rows[c] ? 1 : 0;
    const long long r0 = side == 2 ? -2 : G.nj;
    CUDA_TRY(cudaMemcpyAsync(g->solid + G.soff + r0 * G.ni, h.data(), h.size(), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return ROEAM_OK;
}

extern "C++" {
template <typename T>
static roeam_status set_halo_vertices(roeam_grid *g, const GridDev &G, int side, const double *xv, const double *yv)
{
    std::vector<T> hx(2 * (size_t)G.vpitch, T(0)), hy(2 * (size_t)G.vpitch, T(0));
    const int J0 = side == 2 ? -2 : G.nj + 1;
    for (int r = 0; r < 2; ++r)
        for (int I = 0; I <= G.ni; ++I) {
            const size_t s = (size_t)r * (G.ni + 1) + I;
            hx[(size_t)r * G.vpitch + I] = T(xv[s] - I * G.dx);
            hy[(size_t)r * G.vpitch + I] = T(yv[s] - (J0 + r) * G.dy);
        }
    const size_t at = (size_t)(G.voff + (long long)J0 * G.vpitch);
    CUDA_TRY(cudaMemcpyAsync((T *)g->vdx + at, hx.data(), sizeof(T) * hx.size(), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaMemcpyAsync((T *)g->vdy + at, hy.data(), sizeof(T) * hy.size(), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return ROEAM_OK;
}
}  // extern "C++"

roeam_status roeam_set_halo_vertices(roeam_grid *g, int grid_idx, int side, const double *xv, const double *yv)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (grid_idx < 0) return fail(ROEAM_E_ARG, "ghost rows need one grid (grid_idx >= 0)");
    if (side != 2 && side != 3) return fail(ROEAM_E_ARG, "side must be 2 (S) or 3 (N)");
    const GridDev &G = g->hg[grid_idx];
    if (G.bc[side] != ROEAM_BC_EXCHANGE) return fail(ROEAM_E_ARG, "side %d of grid %d is not EXCHANGE", side, grid_idx);
    if (!g->curv) return fail(ROEAM_E_ARG, "the handle's grids are Cartesian");
    if (!xv || !yv) return fail(ROEAM_E_ARG, "xv and yv must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    return g->precision == 32 ? set_halo_vertices<float>(g, G, side, xv, yv)
                              : set_halo_vertices<double>(g, G, side, xv, yv);
}

roeam_status roeam_math_check(int device, int n, const double *x, double *out)
{
    if (n < 1 || n > (1 << 24) || !x || !out) return fail(ROEAM_E_ARG, "need 1 <= n <= 2^24 and non-null x, out");
    CUDA_TRY(cudaSetDevice(device));
    double *dx = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&dx, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMalloc(&dout, sizeof(double) * 6 * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_math_check(n, dx, dout, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(double) * 6 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(dx);
    cudaFree(dout);
    if (e != cudaSuccess) return fail(ROEAM_E_CUDA, "math check: %s", cudaGetErrorString(e));
    return ROEAM_OK;
}

}  // extern "C"

template <typename H>
static roeam_status step_host(roeam_grid *g, double cfl, double dt_fixed, int nsteps, const H *cons_in, H *cons_out,
                              double *dt_last)
{
    const Range range_("roeam_step_host");
    if (!g || !cons_in || !cons_out) return fail(ROEAM_E_ARG, "null argument");
    if (nsteps < 1) return fail(ROEAM_E_ARG, "nsteps must be >= 1");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail(ROEAM_E_ARG, "need cfl > 0 or dt_fixed > 0");
    if (!std::isfinite(cfl) || !std::isfinite(dt_fixed)) return fail(ROEAM_E_ARG, "cfl and dt_fixed must be finite");
    if (g->stage_next != 0) return fail(ROEAM_E_STATE, "a step run by roeam_rk_stage is unfinished");
    CUDA_TRY(cudaSetDevice(g->device));
    for (int k = 0; k < 3; ++k)
        if (!g->pipe[k]) CUDA_TRY(cudaStreamCreateWithFlags(&g->pipe[k], cudaStreamNonBlocking));
    // chunks of whole grids ending near the cumulative shares of PIPE_SHARES (the last one
    // takes every grid left)
    constexpr int nshares = (int)(sizeof(PIPE_SHARES) / sizeof(PIPE_SHARES[0]));
    double total_share = 0.0;
    for (double x : PIPE_SHARES) total_share += x;
    std::vector<std::pair<int, int>> chunks;
    double cum = 0.0;
    for (int c = 0, lo = 0; c < nshares && lo < g->count; ++c) {
        cum += PIPE_SHARES[c];
        const long long end = (long long)((double)g->total_packed * (cum / total_share));
        int hi = lo + 1;
        while (hi < g->count && g->hg[hi].poff < end) ++hi;
        if (c == nshares - 1) hi = g->count;
        chunks.emplace_back(lo, hi);
        lo = hi;
    }
    if (chunks != g->pipe_chunks || g->pipe_cfg != g->tile_cfg) {
        roeam_status st = setup_pipe_units(g, chunks);
        if (st != ROEAM_OK) return st;
    }
    while (g->pipe_ev.size() < 1 + 2 * chunks.size()) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g->pipe_ev.push_back(e);
    }
    // (the copy engines carry the host data: pack / unpack kernels reading and writing the
    //  page-locked arrays in place measured slower)
    // the three streams start after the work already queued on the handle's stream
    CUDA_TRY(cudaEventRecord(g->pipe_ev[0], g->stream));
    for (int k = 0; k < 3; ++k) CUDA_TRY(cudaStreamWaitEvent(g->pipe[k], g->pipe_ev[0], 0));
    for (size_t c = 0; c < chunks.size(); ++c) {
        const int lo = chunks[c].first, hi = chunks[c].second;
        cudaEvent_t copied = g->pipe_ev[1 + 2 * c], computed = g->pipe_ev[2 + 2 * c];
        roeam_status st =
            g->precision == 32
                ? pipe_chunk<float, H>(g, (int)c, lo, hi, nsteps, cfl, dt_fixed, cons_in, cons_out, copied, computed)
                : pipe_chunk<double, H>(g, (int)c, lo, hi, nsteps, cfl, dt_fixed, cons_in, cons_out, copied, computed);
        if (st != ROEAM_OK) return st;
    }
    // the handle's stream resumes after the last copy out (which follows every computation)
    CUDA_TRY(cudaEventRecord(g->pipe_ev[0], g->pipe[2]));
    CUDA_TRY(cudaStreamWaitEvent(g->stream, g->pipe_ev[0], 0));
    for (int k = 0; k < g->count; ++k) g->state_set[k] = 1;
    const long long step0 = g->step;
    g->step += nsteps;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (dt_last) {
        if (dt_fixed > 0.0) {
            for (int k = 0; k < g->count; ++k) dt_last[k] = dt_fixed;
        } else {
            const int par = (int)((step0 + nsteps - 1) & 1);
            CUDA_TRY(cudaMemcpy(g->h_rate, g->rate + (size_t)par * g->count, sizeof(unsigned long long) * g->count,
                                cudaMemcpyDeviceToHost));
            for (int k = 0; k < g->count; ++k) {
                if (g->precision == 32) {
                    float f;
                    const uint32_t lo32 = (uint32_t)(g->h_rate[k] & 0xffffffffull);
                    std::memcpy(&f, &lo32, sizeof(float));
                    dt_last[k] = (double)(float(cfl) / f);
                } else {
                    double r;
                    std::memcpy(&r, g->h_rate + k, sizeof(double));
                    dt_last[k] = cfl / r;
                }
            }
        }
    }
    return read_status(g);
}

extern "C" {

roeam_status roeam_step_host(roeam_grid *g, double cfl, double dt_fixed, int nsteps, const double *cons_in,
                             double *cons_out, double *dt_last)
{
    return step_host<double>(g, cfl, dt_fixed, nsteps, cons_in, cons_out, dt_last);
}

roeam_status roeam_step_host_f32(roeam_grid *g, double cfl, double dt_fixed, int nsteps, const float *cons_in,
                                 float *cons_out, double *dt_last)
{
    return step_host<float>(g, cfl, dt_fixed, nsteps, cons_in, cons_out, dt_last);
}

roeam_status roeam_set_state_f32(roeam_grid *g, int grid_idx, const float *cons)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (!cons) return fail(ROEAM_E_ARG, "cons must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    return g->precision == 32 ? do_set_state<float, float>(g, grid_idx, cons)
                              : do_set_state<double, float>(g, grid_idx, cons);
}

roeam_status roeam_get_state_f32(roeam_grid *g, int grid_idx, float *cons_out)
{
    roeam_status st = check_idx(g, grid_idx);
    if (st != ROEAM_OK) return st;
    if (!cons_out) return fail(ROEAM_E_ARG, "cons_out must be non-null");
    CUDA_TRY(cudaSetDevice(g->device));
    st = g->precision == 32 ? do_get<float, float>(g, grid_idx, g->U, cons_out)
                            : do_get<double, float>(g, grid_idx, g->U, cons_out);
    if (st != ROEAM_OK) return st;
    return read_status(g);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Residual without device allocation.
//
// Some callers cannot allocate device memory when they need a residual: a host that hands
// the GPU to this library inside a fixed memory budget and forbids allocation after
// start-up, or a monitor that runs next to a solver whose memory pool owns the whole
// device. roeam_flux_residual_noalloc serves them. Its scratch (the residual in working
// precision and its float64 copy) lives in the fixed-size array below, which every GPU that
// loads this library holds until the process exits. Every call shares that array and
// leaves its contents behind; all of it that a call reads is written by the same call
// first, so nothing has to start at zero. Calls whose kernels overlap on the GPU (other
// streams, other threads) race on the array.
namespace {
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(24) << 20;   // 24 MiB
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256] = {nullptr};
}  // namespace

static __device__ __align__(256) unsigned char roeam_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch array on `device` (which must be current). The first call on
// a device (from roeam_create_grid) looks it up with cudaGetSymbolAddress, which loads the
// module and commits the array there; host code may not use the array's name as an address.
roeam_status noalloc_scratch(int device, void **out)
{
    if (device < 0 || device >= 256) return fail(ROEAM_E_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, roeam_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(ROEAM_E_CUDA, "cudaGetSymbolAddress(roeam_noalloc_scratch): %s", cudaGetErrorString(e));
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return ROEAM_OK;
}

template <typename T>
roeam_status do_residual_noalloc(roeam_grid *g, int idx, double *out)
{
    const GridDev &G = g->hg[idx];
    const size_t bytes_t = (sizeof(T) * 4 * (size_t)G.plane + 255) / 256 * 256;
    const size_t bytes_d = sizeof(double) * 4 * (size_t)G.ni * G.nj;
    if (bytes_t + bytes_d > NOALLOC_SCRATCH_BYTES)
        return fail(ROEAM_E_ARG,
                    "grid %d (%d x %d cells) needs %zu bytes of scratch; the allocation-free residual holds %zu "
                    "(about 512 x 512 cells)",
                    idx, G.ni, G.nj, bytes_t + bytes_d, NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    roeam_status st = noalloc_scratch(g->device, &scratch);
    if (st != ROEAM_OK) return st;
    // The kernels address this grid at element offsets G.off (working-precision planes) and
    // G.poff (float64 copy); the shifts place both at the start of their scratch regions.
    T *region_t = (T *)scratch;
    double *region_d = (double *)((unsigned char *)scratch + bytes_t);
    StageArgs<T> a = base_args<T>(g);
    a.mode = MODE_RESIDUAL;
    a.src = (const T *)g->U;
    a.un = (const T *)g->U;
    a.dst = region_t;
    a.dst_shift = G.off;
#ifdef ROEAM_DEBUG
    a.n_dst = 4 * G.plane;
#endif
    a.units = g->d_units_grid;
    a.tile_lo = g->h_tile_base[idx];
    a.tile_hi = g->h_tile_base[idx + 1];
    CUDA_TRY(Launchers<T>::stage(a, g->muscl, g->curv, g->kind, g->nblocks, g->stream));
    CUDA_TRY(Launchers<T>::unpack(g->d_grids, idx, idx + 1, G.ni * G.nj, region_t, region_d, g->stream, G.off,
                                  G.poff));
    g->launches += 2;
    CUDA_TRY(cudaMemcpyAsync(out, region_d, bytes_d, cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return ROEAM_OK;
}

}  // namespace

extern "C" roeam_status roeam_flux_residual_noalloc(roeam_grid *g, int grid_idx, double *res_out)
{
    if (!g) return fail(ROEAM_E_ARG, "null handle");
    if (grid_idx < 0 || grid_idx >= g->count) return fail(ROEAM_E_ARG, "grid_idx %d out of range [0, %d)", grid_idx, g->count);
    if (!res_out) return fail(ROEAM_E_ARG, "res_out must be non-null");
    if (!g->state_set[grid_idx]) return fail(ROEAM_E_STATE, "state of grid %d not set", grid_idx);
    CUDA_TRY(cudaSetDevice(g->device));
    return g->precision == 32 ? do_residual_noalloc<float>(g, grid_idx, res_out)
                              : do_residual_noalloc<double>(g, grid_idx, res_out);
}
