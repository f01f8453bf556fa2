// roeam3_api.cu — host implementation of the 3D C ABI declared in include/roeam3.h.
//
// Owns the device memory of a batch of 3D grids (pitched structure-of-arrays volumes, one per
// conserved variable), builds the work units of the 3D stage kernel (30 x 14 columns of a plane
// in FP32, 30 x 6 in FP64, by a segment of planes), and drives the three fused stage launches of each SSP-RK3 step with
// per-grid time steps read on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "roeam.h"
#include "roeam3.h"
#include "roeam3_internal.h"

using namespace roeam;

namespace {

roeam_status fail3(roeam_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return (roeam_status)record_error(st, buf);
}

#define CUDA_TRY3(expr)                                                                                      \
    do {                                                                                                     \
        cudaError_t e_ = (expr);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return fail3(e_ == cudaErrorMemoryAllocation ? ROEAM_E_OOM : ROEAM_E_CUDA, "%s: %s (%s:%d)", #expr, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                                        \
    } while (0)

long long round_up3(long long a, long long m) { return (a + m - 1) / m * m; }

}  // namespace

struct roeam3_grid {
    int device = 0;
    cudaStream_t stream = nullptr;
    int precision = 32, nscal = 0, nv = 5, count = 0;
    size_t esize = 4;
    std::vector<GridDev3> hg;
    GridDev3 *d_grids = nullptr;
    void *d_coef = nullptr;
    void *U = nullptr, *A = nullptr, *B = nullptr;
    long long total_elems = 0, total_packed = 0, max_cells = 0;
    int4 *d_units = nullptr;
    int nunits = 0, nblocks = 0;
    unsigned long long *rate = nullptr;   // 2 x count slots, alternating by step parity
    int parity = 0;
    unsigned *status = nullptr;
    double *staging = nullptr;            // float64 packed copy on the device
    double *partials = nullptr;
    double *h_red = nullptr;              // pinned
    unsigned *h_status = nullptr;         // pinned
    unsigned long long *h_rate = nullptr; // pinned
    unsigned long long launches = 0;
};

namespace {

roeam_status validate3(int count, const roeam3_grid_desc *d)
{
    if (count < 1 || !d) return fail3(ROEAM_E_ARG, "count must be >= 1 and descs non-null");
    if (count > 65535) return fail3(ROEAM_E_ARG, "count must be <= 65535 grids per handle");
    for (int k = 0; k < count; ++k) {
        const roeam3_grid_desc &q = d[k];
        const roeam_params &p = q.p;
        if (q.ni < 1 || q.nj < 1 || q.nk < 1 || q.ni > 65535 || q.nj > 65535 || q.nk > 65535)
            return fail3(ROEAM_E_ARG, "grid %d: ni, nj, nk must be in 1..65535", k);
        if ((long long)q.ni * q.nj * q.nk > (1ll << 28)) return fail3(ROEAM_E_ARG, "grid %d: too many cells", k);
        if (!(q.dx > 0.0) || !(q.dy > 0.0) || !(q.dz > 0.0)) return fail3(ROEAM_E_ARG, "grid %d: dx, dy, dz must be > 0", k);
        if (q.nscal < 0 || q.nscal > ROEAM3_MAX_SCALARS) return fail3(ROEAM_E_ARG, "grid %d: nscal must be 0..3", k);
        if (q.nscal != d[0].nscal) return fail3(ROEAM_E_ARG, "grid %d: nscal differs within the batch", k);
        if (q.reserved_ != 0) return fail3(ROEAM_E_ARG, "grid %d: reserved_ must be 0", k);
        if (!(p.gamma > 1.0)) return fail3(ROEAM_E_ARG, "grid %d: gamma must be > 1", k);
        if (!(p.m_ref > 0.0)) return fail3(ROEAM_E_ARG, "grid %d: m_ref must be > 0", k);
        if (!(p.u_ref > 0.0)) return fail3(ROEAM_E_ARG, "grid %d: u_ref must be > 0", k);
        if (!(p.eps2 >= 0.0)) return fail3(ROEAM_E_ARG, "grid %d: eps2 must be >= 0", k);
        if (p.eps1 != 0 && p.eps1 != 1) return fail3(ROEAM_E_ARG, "grid %d: eps1 must be 0 or 1", k);
        if (p.use_s1 != 0 && p.use_s1 != 1) return fail3(ROEAM_E_ARG, "grid %d: use_s1 must be 0 or 1", k);
        if (p.xi_form != 0 && p.xi_form != 1) return fail3(ROEAM_E_ARG, "grid %d: xi_form must be 0 or 1", k);
        if (p.recon != ROEAM_RECON_FIRST) return fail3(ROEAM_E_ARG, "grid %d: the 3D path is first order (recon 0)", k);
        if (p.scheme || p.dup_mode || p.no_ufix || p.xi_roe || p.harten != 0.0 || p.reserved_)
            return fail3(ROEAM_E_ARG, "grid %d: the 3D path has no ablation variants", k);
        if (p.precision != 32 && p.precision != 64) return fail3(ROEAM_E_ARG, "grid %d: precision must be 32 or 64", k);
        if (p.precision != d[0].p.precision) return fail3(ROEAM_E_ARG, "grid %d: precision differs within the batch", k);
        for (int s = 0; s < 6; ++s)
            if (q.bc[s] < 0 || q.bc[s] > 3) return fail3(ROEAM_E_ARG, "grid %d: bad boundary type on side %d", k, s);
        for (int a = 0; a < 3; ++a)
            if ((q.bc[2 * a] == ROEAM_BC_PERIODIC) != (q.bc[2 * a + 1] == ROEAM_BC_PERIODIC))
                return fail3(ROEAM_E_ARG, "grid %d: PERIODIC must be set on both sides of axis %d", k, a);
        for (int s = 0; s < 6; ++s)
            if (q.bc[s] == ROEAM_BC_INFLOW && !(q.inflow[0] > 0.0 && q.inflow[4] > 0.0))
                return fail3(ROEAM_E_ARG, "grid %d: inflow density and pressure must be > 0", k);
    }
    return ROEAM_OK;
}

template <typename T>
roeam_status upload_coef3(roeam3_grid *g, const roeam3_grid_desc *d)
{
    std::vector<GridCoef3<T>> h(g->count);
    for (int k = 0; k < g->count; ++k) {
        const roeam3_grid_desc &q = d[k];
        GridCoef3<T> &c = h[k];
        const double gm = q.p.gamma;
        c.g = T(gm);
        c.gm1 = T(gm - 1.0);
        c.gm1i = T(1.0 / (gm - 1.0));
        c.hgm1 = T(0.5 * (gm - 1.0));
        c.mr2 = T(q.p.m_ref * q.p.m_ref);
        c.rr_thr = T(1e-5 * q.p.u_ref);
        c.eps2 = T(q.p.eps2);
        c.ax = T(q.dy * q.dz);
        c.ay = T(q.dx * q.dz);
        c.az = T(q.dx * q.dy);
        c.Vi = T(1.0 / (q.dx * q.dy * q.dz));
        c.idx = T(1.0 / q.dx);
        c.idy = T(1.0 / q.dy);
        c.idz = T(1.0 / q.dz);
        for (int v = 0; v < MAX_VARS3; ++v) c.inflow[v] = T(q.inflow[v]);
    }
    CUDA_TRY3(cudaMalloc(&g->d_coef, sizeof(GridCoef3<T>) * g->count));
    CUDA_TRY3(cudaMemcpy(g->d_coef, h.data(), sizeof(GridCoef3<T>) * g->count, cudaMemcpyHostToDevice));
    return ROEAM_OK;
}

// Work units: 30 x 14 columns of a plane in FP32, 30 x 6 in FP64 (TILE3_X x tile3_y<T>() written
// cells) by a segment of
// planes. The number of segments per column starts at about four units per resident CTA and is
// then chosen, up to twice that, to fill the last round of units over the CTAs (all units cost
// about the same): the 256^3 Taylor-Green vortex had 1548 units over 304 CTAs, a sixth round
// 9 % full; 7 segments give 2709 units in 8.9 rounds. Each extra segment re-reads two planes,
// which the choice weighs at half a plane of work each.
roeam_status setup_units3(roeam3_grid *g, int num_sms)
{
    const int occ = g->precision == 32 ? Launchers3<float>::stage_occupancy(g->nscal)
                                       : Launchers3<double>::stage_occupancy(g->nscal);
    g->nblocks = std::max(1, occ * num_sms);
    const int TILE3_Y = g->precision == 32 ? tile3_y<float>() : tile3_y<double>();
    long long columns = 0, nk_max = 1;
    for (const GridDev3 &G : g->hg) {
        columns += (long long)((G.ni + TILE3_X - 1) / TILE3_X) * ((G.nj + TILE3_Y - 1) / TILE3_Y);
        nk_max = std::max<long long>(nk_max, G.nk);
    }
    const long long target = 4ll * g->nblocks;
    const long long nseg0 = std::max(1ll, (target + columns - 1) / columns);
    long long nseg = nseg0;
    {
        double best = -1.0;
        for (long long n = nseg0; n <= 2 * nseg0; ++n) {
            long long units = 0;
            double planes = 0.0, extra = 0.0;
            for (const GridDev3 &G : g->hg) {
                const long long cols = (long long)((G.ni + TILE3_X - 1) / TILE3_X) * ((G.nj + TILE3_Y - 1) / TILE3_Y);
                const int zs = std::max(4, (int)((G.nk + n - 1) / n));
                const long long segs = (G.nk + zs - 1) / zs;
                units += cols * segs;
                planes += (double)cols * G.nk;
                extra += (double)cols * segs;   // two re-read planes per segment, at half a plane each
            }
            const long long rounds = (units + g->nblocks - 1) / g->nblocks;
            const double eff = (double)units / (double)(rounds * g->nblocks) * planes / (planes + extra);
            if (eff > best + 1e-9) { best = eff; nseg = n; }
        }
    }
    std::vector<int4> units;
    for (int gi = 0; gi < g->count; ++gi) {
        const GridDev3 &G = g->hg[gi];
        const int zs = std::max(4, (int)((G.nk + nseg - 1) / nseg));
        for (int k0 = 0; k0 < G.nk; k0 += zs) {
            const int k1 = std::min(G.nk, k0 + zs);
            for (int j0 = 0; j0 < G.nj; j0 += TILE3_Y)
                for (int i0 = 0; i0 < G.ni; i0 += TILE3_X) units.push_back(make_int4(gi, i0, j0, k0 | (k1 << 16)));
        }
    }
    g->nunits = (int)units.size();
    g->nblocks = (int)std::min<long long>(g->nblocks, g->nunits);
    CUDA_TRY3(cudaMalloc(&g->d_units, sizeof(int4) * units.size()));
    CUDA_TRY3(cudaMemcpy(g->d_units, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice));
    return ROEAM_OK;
}

template <typename T>
StageArgs3<T> base_args3(roeam3_grid *g)
{
    StageArgs3<T> a;
    std::memset(&a, 0, sizeof(a));
    a.grids = g->d_grids;
    a.coef = (const GridCoef3<T> *)g->d_coef;
    a.units = g->d_units;
    a.ngrids = g->count;
    a.nunits = g->nunits;
    a.status = g->status;
    return a;
}

template <typename T>
roeam_status refresh_rate3(roeam3_grid *g)
{
    unsigned long long *slot = g->rate + (size_t)g->parity * g->count;
    CUDA_TRY3(cudaMemsetAsync(slot, 0, sizeof(unsigned long long) * g->count, g->stream));
    CUDA_TRY3(Launchers3<T>::rate(g->d_grids, (const GridCoef3<T> *)g->d_coef, 0, g->count, (const T *)g->U, g->nscal,
                                  slot, g->stream));
    g->launches += 1;
    return ROEAM_OK;
}

template <typename T>
roeam_status do_set3(roeam3_grid *g, int lo, int hi, const double *host)
{
    const GridDev3 &a = g->hg[lo], &b = g->hg[hi - 1];
    const long long n0 = a.poff, n1 = b.poff + (long long)g->nv * b.ni * b.nj * b.nk;
    CUDA_TRY3(cudaMemcpyAsync(g->staging + n0, host, sizeof(double) * (n1 - n0), cudaMemcpyHostToDevice, g->stream));
    CUDA_TRY3(Launchers3<T>::pack(g->d_grids, lo, hi, g->nv, g->max_cells, g->staging, (T *)g->U, g->stream));
    g->launches += 1;
    return refresh_rate3<T>(g);
}

roeam_status sync_status3(roeam3_grid *g)
{
    CUDA_TRY3(cudaMemcpyAsync(g->h_status, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY3(cudaMemsetAsync(g->status, 0, sizeof(unsigned), g->stream));
    CUDA_TRY3(cudaStreamSynchronize(g->stream));
    const unsigned st = *g->h_status;
    if (st & ST_NONFINITE) return fail3(ROEAM_E_NONFINITE, "non-finite state after a step");
    if (st & ST_NONPOSITIVE) return fail3(ROEAM_E_NONPOSITIVE, "non-positive density or pressure after a step");
    return ROEAM_OK;
}

template <typename T>
roeam_status do_get3(roeam3_grid *g, int lo, int hi, double *host, const void *src)
{
    CUDA_TRY3(Launchers3<T>::unpack(g->d_grids, lo, hi, g->nv, g->max_cells, (const T *)src, g->staging, g->stream));
    g->launches += 1;
    const GridDev3 &a = g->hg[lo], &b = g->hg[hi - 1];
    const long long n0 = a.poff, n1 = b.poff + (long long)g->nv * b.ni * b.nj * b.nk;
    CUDA_TRY3(cudaMemcpyAsync(host, g->staging + n0, sizeof(double) * (n1 - n0), cudaMemcpyDeviceToHost, g->stream));
    return sync_status3(g);
}

template <typename T>
roeam_status launch_step3(roeam3_grid *g, double cfl, double dt_fixed)
{
    StageArgs3<T> a = base_args3<T>(g);
    a.cfl_t = T(cfl);
    a.dt_fixed_t = T(dt_fixed);
    a.mode = MODE_STAGE;
    a.rate_rd = g->rate + (size_t)g->parity * g->count;
    a.rate_wr = g->rate + (size_t)(1 - g->parity) * g->count;
    const T *U = (const T *)g->U;
    // stage 1: U1 = U + dt R(U)   (also clears the next step's rate slots)
    a.src = U; a.un = U; a.dst = (T *)g->A; a.alpha = T(0); a.beta = T(1); a.rate_zero = a.rate_wr; a.want_rate = 0;
    CUDA_TRY3(Launchers3<T>::stage(a, g->nscal, g->nblocks, g->stream));
    // stage 2: U2 = 3/4 U + 1/4 (U1 + dt R(U1))
    a.src = (const T *)g->A; a.dst = (T *)g->B; a.alpha = T(0.75); a.beta = T(0.25); a.rate_zero = nullptr;
    CUDA_TRY3(Launchers3<T>::stage(a, g->nscal, g->nblocks, g->stream));
    // stage 3: U = 1/3 U + 2/3 (U2 + dt R(U2)), in place; the next step's rate
    a.src = (const T *)g->B; a.dst = (T *)g->U; a.alpha = T(1.0 / 3.0); a.beta = T(2.0 / 3.0); a.want_rate = 1;
    CUDA_TRY3(Launchers3<T>::stage(a, g->nscal, g->nblocks, g->stream));
    g->launches += 3;
    g->parity ^= 1;
    return ROEAM_OK;
}

template <typename T>
roeam_status do_residual3(roeam3_grid *g, int lo, int hi, double *out)
{
    StageArgs3<T> a = base_args3<T>(g);
    a.mode = MODE_RESIDUAL;
    a.src = (const T *)g->U;
    a.un = (const T *)g->U;
    a.dst = (T *)g->A;
    CUDA_TRY3(Launchers3<T>::stage(a, g->nscal, g->nblocks, g->stream));
    g->launches += 1;
    if (!out) return ROEAM_OK;
    return do_get3<T>(g, lo, hi, out, g->A);
}

template <typename T>
roeam_status do_totals3(roeam3_grid *g, int idx, double *out)
{
    const GridDev3 &G = g->hg[idx];
    const long long n = (long long)G.ni * G.nj * G.nk;
    const int nb = (int)std::min<long long>((n + 255) / 256, 1024);
    CUDA_TRY3(Launchers3<T>::totals(g->d_grids, idx, (const T *)g->U, g->nv, g->partials, nb, g->stream));
    g->launches += 1;
    std::vector<double> h((size_t)nb * MAX_VARS3);
    CUDA_TRY3(cudaMemcpyAsync(h.data(), g->partials, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY3(cudaStreamSynchronize(g->stream));
    for (int v = 0; v < g->nv; ++v) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += h[(size_t)b * MAX_VARS3 + v];   // fixed order
        out[v] = s;
    }
    return ROEAM_OK;
}

roeam_status range3(roeam3_grid *g, int idx, int &lo, int &hi)
{
    if (!g) return fail3(ROEAM_E_ARG, "null handle");
    if (idx < -1 || idx >= g->count) return fail3(ROEAM_E_ARG, "grid index %d out of range", idx);
    lo = idx < 0 ? 0 : idx;
    hi = idx < 0 ? g->count : idx + 1;
    if (cudaSetDevice(g->device) != cudaSuccess) return fail3(ROEAM_E_CUDA, "cudaSetDevice failed");
    return ROEAM_OK;
}

}  // namespace

extern "C" {

roeam_status roeam3_create_grid(int count, const roeam3_grid_desc *descs, int device, void *cuda_stream,
                                roeam3_grid **out)
{
    if (!out) return fail3(ROEAM_E_ARG, "out must be non-null");
    *out = nullptr;
    roeam_status st = validate3(count, descs);
    if (st != ROEAM_OK) return st;
    CUDA_TRY3(cudaSetDevice(device));
    int num_sms = 0;
    CUDA_TRY3(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
    roeam3_grid *g = new roeam3_grid();
    g->device = device;
    g->stream = (cudaStream_t)cuda_stream;
    g->count = count;
    g->precision = descs[0].p.precision;
    g->esize = g->precision == 32 ? 4 : 8;
    g->nscal = descs[0].nscal;
    g->nv = 5 + g->nscal;
    g->hg.resize(count);
    long long off = 0, poff = 0;
    for (int k = 0; k < count; ++k) {
        const roeam3_grid_desc &q = descs[k];
        GridDev3 &G = g->hg[k];
        std::memset(&G, 0, sizeof(G));
        G.ni = q.ni; G.nj = q.nj; G.nk = q.nk;
        G.pitch = (int)round_up3(q.ni, 32);
        G.vol = (long long)q.nk * q.nj * G.pitch;
        G.off = off;
        off += round_up3((long long)g->nv * G.vol, 64);
        G.poff = poff;
        poff += (long long)g->nv * q.ni * q.nj * q.nk;
        for (int s = 0; s < 6; ++s) G.bc[s] = q.bc[s];
        G.eps1 = q.p.eps1; G.use_s1 = q.p.use_s1; G.xi_form = q.p.xi_form;
        for (int v = 0; v < MAX_VARS3; ++v) G.inflow[v] = q.inflow[v];
        G.gamma = q.p.gamma; G.m_ref = q.p.m_ref; G.u_ref = q.p.u_ref; G.eps2 = q.p.eps2;
        G.dx = q.dx; G.dy = q.dy; G.dz = q.dz;
        g->max_cells = std::max(g->max_cells, (long long)q.ni * q.nj * q.nk);
    }
    g->total_elems = off;
    g->total_packed = poff;
    auto cleanup = [&](roeam_status s) { roeam3_destroy_grid(g); return s; };
#define CREATE3_TRY(expr)                                                                                        \
    do {                                                                                                         \
        cudaError_t e_ = (expr);                                                                                 \
        if (e_ != cudaSuccess)                                                                                   \
            return cleanup(fail3(e_ == cudaErrorMemoryAllocation ? ROEAM_E_OOM : ROEAM_E_CUDA, "%s: %s", #expr, \
                                 cudaGetErrorString(e_)));                                                       \
    } while (0)
    const size_t sbytes = g->esize * (size_t)g->total_elems;
    CREATE3_TRY(cudaMalloc(&g->U, sbytes));
    CREATE3_TRY(cudaMalloc(&g->A, sbytes));
    CREATE3_TRY(cudaMalloc(&g->B, sbytes));
    CREATE3_TRY(cudaMemset(g->U, 0, sbytes));
    CREATE3_TRY(cudaMemset(g->A, 0, sbytes));
    CREATE3_TRY(cudaMemset(g->B, 0, sbytes));
    CREATE3_TRY(cudaMalloc(&g->d_grids, sizeof(GridDev3) * count));
    CREATE3_TRY(cudaMemcpy(g->d_grids, g->hg.data(), sizeof(GridDev3) * count, cudaMemcpyHostToDevice));
    CREATE3_TRY(cudaMalloc(&g->rate, sizeof(unsigned long long) * 2 * count));
    CREATE3_TRY(cudaMemset(g->rate, 0, sizeof(unsigned long long) * 2 * count));
    CREATE3_TRY(cudaMalloc(&g->status, sizeof(unsigned)));
    CREATE3_TRY(cudaMemset(g->status, 0, sizeof(unsigned)));
    CREATE3_TRY(cudaMalloc(&g->staging, sizeof(double) * (size_t)std::max(1ll, g->total_packed)));
    CREATE3_TRY(cudaMalloc(&g->partials, sizeof(double) * 1024 * MAX_VARS3));
    CREATE3_TRY(cudaMallocHost(&g->h_status, sizeof(unsigned)));
    CREATE3_TRY(cudaMallocHost(&g->h_rate, sizeof(unsigned long long) * count));
#undef CREATE3_TRY
    st = g->precision == 32 ? upload_coef3<float>(g, descs) : upload_coef3<double>(g, descs);
    if (st != ROEAM_OK) return cleanup(st);
    st = setup_units3(g, num_sms);
    if (st != ROEAM_OK) return cleanup(st);
    *out = g;
    return ROEAM_OK;
}

void roeam3_destroy_grid(roeam3_grid *g)
{
    if (!g) return;
    cudaSetDevice(g->device);
    if (g->stream) cudaStreamSynchronize(g->stream); else cudaDeviceSynchronize();
    cudaFree(g->U); cudaFree(g->A); cudaFree(g->B);
    cudaFree(g->d_grids); cudaFree(g->d_coef); cudaFree(g->d_units);
    cudaFree(g->rate); cudaFree(g->status); cudaFree(g->staging); cudaFree(g->partials);
    cudaFreeHost(g->h_status); cudaFreeHost(g->h_rate);
    delete g;
}

roeam_status roeam3_set_state(roeam3_grid *g, int grid_idx, const double *cons)
{
    int lo, hi;
    roeam_status st = range3(g, grid_idx, lo, hi);
    if (st != ROEAM_OK) return st;
    if (!cons) return fail3(ROEAM_E_ARG, "cons must be non-null");
    return g->precision == 32 ? do_set3<float>(g, lo, hi, cons) : do_set3<double>(g, lo, hi, cons);
}

roeam_status roeam3_get_state(roeam3_grid *g, int grid_idx, double *cons_out)
{
    int lo, hi;
    roeam_status st = range3(g, grid_idx, lo, hi);
    if (st != ROEAM_OK) return st;
    if (!cons_out) return fail3(ROEAM_E_ARG, "cons_out must be non-null");
    return g->precision == 32 ? do_get3<float>(g, lo, hi, cons_out, g->U) : do_get3<double>(g, lo, hi, cons_out, g->U);
}

roeam_status roeam3_flux_residual(roeam3_grid *g, int grid_idx, double *res_out)
{
    int lo, hi;
    roeam_status st = range3(g, grid_idx, lo, hi);
    if (st != ROEAM_OK) return st;
    return g->precision == 32 ? do_residual3<float>(g, lo, hi, res_out) : do_residual3<double>(g, lo, hi, res_out);
}

roeam_status roeam3_rk_step(roeam3_grid *g, double cfl, double dt_fixed, int nsteps, double *dt_last)
{
    int lo, hi;
    roeam_status st = range3(g, -1, lo, hi);
    if (st != ROEAM_OK) return st;
    if (nsteps < 0) return fail3(ROEAM_E_ARG, "nsteps must be >= 0");
    if (!(dt_fixed > 0.0) && !(cfl > 0.0)) return fail3(ROEAM_E_ARG, "give cfl > 0 or dt_fixed > 0");
    for (int s = 0; s < nsteps; ++s) {
        st = g->precision == 32 ? launch_step3<float>(g, cfl, dt_fixed) : launch_step3<double>(g, cfl, dt_fixed);
        if (st != ROEAM_OK) return st;
    }
    if (dt_last) {
        if (dt_fixed > 0.0 || nsteps == 0) {
            for (int k = 0; k < g->count; ++k) dt_last[k] = nsteps == 0 ? 0.0 : dt_fixed;
        } else {
            // the last step read the slots of the parity before the flip
            const unsigned long long *slot = g->rate + (size_t)(g->parity ^ 1) * g->count;
            CUDA_TRY3(cudaMemcpyAsync(g->h_rate, slot, sizeof(unsigned long long) * g->count, cudaMemcpyDeviceToHost,
                                      g->stream));
            st = sync_status3(g);
            if (st != ROEAM_OK) return st;
            for (int k = 0; k < g->count; ++k) {
                if (g->precision == 32) {
                    float f;
                    const unsigned bits = (unsigned)g->h_rate[k];
                    std::memcpy(&f, &bits, 4);
                    dt_last[k] = (double)(float(cfl) / f);
                } else {
                    double r;
                    std::memcpy(&r, &g->h_rate[k], 8);
                    dt_last[k] = cfl / r;
                }
            }
        }
    }
    return ROEAM_OK;
}

roeam_status roeam3_conserved_totals(roeam3_grid *g, int grid_idx, double *out)
{
    int lo, hi;
    if (grid_idx < 0) return fail3(ROEAM_E_ARG, "grid_idx must be >= 0");
    roeam_status st = range3(g, grid_idx, lo, hi);
    if (st != ROEAM_OK) return st;
    if (!out) return fail3(ROEAM_E_ARG, "out must be non-null");
    st = sync_status3(g);
    if (st != ROEAM_OK) return st;
    return g->precision == 32 ? do_totals3<float>(g, grid_idx, out) : do_totals3<double>(g, grid_idx, out);
}

roeam_status roeam3_check(roeam3_grid *g)
{
    int lo, hi;
    roeam_status st = range3(g, -1, lo, hi);
    if (st != ROEAM_OK) return st;
    return sync_status3(g);
}

unsigned long long roeam3_launch_count(const roeam3_grid *g) { return g ? g->launches : 0ull; }

}  // extern "C"
