// Ensembles of independent problems advanced together (host side of the C
// ABI's rkl_ensemble_* entry points).  One super-step of every problem is
// either one persistent launch of a tile body (paired-cell or row-pair)
// over a stage-major work list (default) or, as the alternative schedule,
// one kernel launch per problem and stage.  Problems keep their own grid size,
// conductivity, super-step and stage count.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rkl.h"
#include "rkl_launch.h"
#include "rkl_x2.cuh"

using namespace rkl;

namespace rkl {
void set_unplanned_error(const std::string& msg);
}

namespace {
constexpr int kChunk = 65536;            // cells per statistics chunk
}  // namespace

struct rkl_ensemble {
    int nprob = 0;
    std::vector<rkl_grid> grid;
    std::vector<rkl_phys> phys;
    std::vector<KGrid<float>> kg;
    std::vector<KPhys<float>> kp;
    std::vector<int64_t> off;            // cell offsets, nprob + 1 entries (multiples of 4)
    int64_t total = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool spitzer = false, saturate = false;

    float* ws = nullptr;                 // 4 * total floats: buf0, buf1, buf2, M(Y0)
    int nchunk = 0;
    int64_t* d_cstart = nullptr;
    int* d_clen = nullptr;
    int* d_pchunk = nullptr;
    double* d_partials = nullptr;
    double* d_pstats = nullptr;          // [nprob][3]
    double* h_pstats = nullptr;          // pinned

    x2::EnsProb* d_probs = nullptr;
    x2::EnsProb* h_probs = nullptr;      // pinned
    x2::EnsSeg* d_segs = nullptr;
    x2::EnsSeg* h_segs = nullptr;        // pinned
    int seg_cap = 0;
    float* d_coef = nullptr;
    float* h_coef = nullptr;             // pinned
    int coef_cap = 0;
    int* d_work = nullptr;
    unsigned* d_done = nullptr;
    int* d_abort = nullptr;
    unsigned* d_status = nullptr;
    unsigned* h_status = nullptr;        // pinned

    int persistent = 1;                  // schedule: bit 0 persistent launch, bit 1 row-pair tiles
    int nzchunk = 32;
    bool rowpair_ok = true;              // every problem periodic with < 2^31 cells
    long long spin_limit = 20000000;     // ~ a few seconds of bounded waiting
    std::vector<int> last_s;
    std::string err;
};

namespace {

// Tile width and counts of one problem: 32-column tiles where they cover
// the width with fewer idle columns than 64-column ones (nx an odd
// multiple of 32, e.g. 32 or 96), else 64-column tiles.  Paired-cell tiles
// are 4 (64 columns) or 8 (32 columns) rows high, row-pair tiles 8 or 16.
void set_tiles(x2::EnsProb& d, int nzchunk, bool rowpair)
{
    const int nx = d.g.n[0];
    const bool narrow = (nx + 31) / 32 * 32 < (nx + 63) / 64 * 64;
    d.txw = narrow ? 32 : x2::TX;
    const int tyh = (rowpair ? 2 : 1) * x2::NTHREADS / (d.txw / 2);
    d.tx = (nx + d.txw - 1) / d.txw;
    d.ty = (d.g.n[1] + tyh - 1) / tyh;
    d.tz = (d.g.n[2] + nzchunk - 1) / nzchunk;
    d.ntiles = d.tx * d.ty * d.tz;
}

rkl_status efail(rkl_ensemble* e, rkl_status st, const std::string& m)
{
    if (e) e->err = m;
    else rkl::set_unplanned_error(m);
    return st;
}

#define ENS_CK(e, call)                                                                          \
    do {                                                                                         \
        cudaError_t c_ = (call);                                                                 \
        if (c_ != cudaSuccess) return efail((e), RKL_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(c_)); \
    } while (0)

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

struct Guard {
    int prev = -1;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~Guard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

double kpar_host(const rkl_phys& ph, double T)
{
    return ph.kappa_model == RKL_KAPPA_SPITZER ? ph.kappa_par0 * T * T * std::sqrt(T) : ph.kappa_par0;
}

template <typename T>
rkl_status grow_pinned(rkl_ensemble* e, T** d, T** h, int* cap, int need)
{
    if (need <= *cap) return RKL_OK;
    int ncap = std::max(need, *cap * 2);
    if (*d) cudaFree(*d);
    if (*h) cudaFreeHost(*h);
    *d = nullptr;
    *h = nullptr;
    ENS_CK(e, cudaMalloc(d, sizeof(T) * ncap));
    ENS_CK(e, cudaMallocHost(h, sizeof(T) * ncap));
    *cap = ncap;
    return RKL_OK;
}

// Per-problem statistics of T_all into h_pstats (synchronises); also reads
// and clears the ensemble's device status word.
rkl_status ens_stats(rkl_ensemble* e, const float* T_all)
{
    cudaError_t c = launch_stats_segmented(T_all, e->d_cstart, e->d_clen, e->nchunk, e->d_pchunk, e->nprob,
                                           e->d_partials, e->d_pstats, e->stream);
    if (c != cudaSuccess) return efail(e, RKL_ERR_CUDA, std::string("stats: ") + cudaGetErrorString(c));
    ENS_CK(e, cudaMemcpyAsync(e->h_pstats, e->d_pstats, sizeof(double) * 3 * e->nprob, cudaMemcpyDeviceToHost,
                              e->stream));
    ENS_CK(e, cudaMemcpyAsync(e->h_status, e->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_status, 0, sizeof(unsigned), e->stream));
    ENS_CK(e, cudaStreamSynchronize(e->stream));
    const unsigned w = *e->h_status;
    if (w & ST_NONFINITE) return efail(e, RKL_ERR_NONFINITE, "a stage produced NaN or Inf");
    if (w & ST_NONPOSITIVE) return efail(e, RKL_ERR_NONPOSITIVE_T, "a stage produced T <= 0 under Spitzer kappa");
    if (w & ST_TIMEOUT) return efail(e, RKL_ERR_TIMEOUT, "a bounded wait of the persistent kernel gave up");
    return RKL_OK;
}

// One super-step of every problem with the given stage counts.
rkl_status ens_run(rkl_ensemble* e, const double* dt, const int* s, float* T_all, const float* b_all)
{
    const int np = e->nprob;
    // coefficient tables, FP64 -> FP32, stage j of problem p at coef[cofs[p] + 4 j]
    std::vector<int> cofs(np + 1, 0);
    for (int p = 0; p < np; ++p) cofs[p + 1] = cofs[p] + 4 * (s[p] + 1);
    rkl_status st = grow_pinned(e, &e->d_coef, &e->h_coef, &e->coef_cap, cofs[np]);
    if (st != RKL_OK) return st;
    std::vector<double> mu, nu, mut, gt;
    int smax = 0, total_items = 0;
    for (int p = 0; p < np; ++p) {
        mu.assign(s[p] + 1, 0.0); nu = mu; mut = mu; gt = mu;
        rkl_coeffs(s[p], mu.data(), nu.data(), mut.data(), gt.data());
        float* h = e->h_coef + cofs[p];
        for (int j = 0; j <= s[p]; ++j) {
            h[4 * j + 0] = (float)mu[j];
            h[4 * j + 1] = (float)nu[j];
            h[4 * j + 2] = (float)(mut[j] * dt[p]);
            h[4 * j + 3] = (float)(gt[j] * dt[p]);
        }
        smax = std::max(smax, s[p]);
        x2::EnsProb& d = e->h_probs[p];
        d.g = e->kg[p];
        d.p = e->kp[p];
        d.T = T_all + e->off[p];
        d.b = b_all + 3 * e->off[p];
        for (int k = 0; k < 3; ++k) d.buf[k] = e->ws + (int64_t)k * e->total + e->off[p];
        d.my0 = e->ws + 3 * e->total + e->off[p];
        d.coef = e->d_coef + cofs[p];
        d.s = s[p];
        d.nzchunk = e->nzchunk;
        set_tiles(d, e->nzchunk, (e->persistent & 2) != 0);
        total_items += d.ntiles * s[p];
    }
    ENS_CK(e, cudaMemcpyAsync(e->d_coef, e->h_coef, sizeof(float) * cofs[np], cudaMemcpyHostToDevice, e->stream));
    if (e->persistent & 1) {
        // stage-major work list
        int nseg = 0;
        for (int j = 1; j <= smax; ++j)
            for (int p = 0; p < np; ++p)
                if (s[p] >= j) ++nseg;
        st = grow_pinned(e, &e->d_segs, &e->h_segs, &e->seg_cap, nseg);
        if (st != RKL_OK) return st;
        int item = 0, k = 0;
        for (int j = 1; j <= smax; ++j)
            for (int p = 0; p < np; ++p)
                if (s[p] >= j) {
                    e->h_segs[k++] = x2::EnsSeg{item, p, j, e->h_probs[p].ntiles};
                    item += e->h_probs[p].ntiles;
                }
        ENS_CK(e, cudaMemcpyAsync(e->d_probs, e->h_probs, sizeof(x2::EnsProb) * np, cudaMemcpyHostToDevice,
                                  e->stream));
        ENS_CK(e, cudaMemcpyAsync(e->d_segs, e->h_segs, sizeof(x2::EnsSeg) * nseg, cudaMemcpyHostToDevice,
                                  e->stream));
        ENS_CK(e, cudaMemsetAsync(e->d_work, 0, sizeof(int), e->stream));
        ENS_CK(e, cudaMemsetAsync(e->d_abort, 0, sizeof(int), e->stream));
        ENS_CK(e, cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * np, e->stream));
        cudaError_t c = (e->persistent & 2)
                            ? launch_ensemble_xq(e->spitzer, e->saturate, e->d_probs, e->d_segs, nseg, total_items,
                                                 e->d_work, e->d_done, e->d_status, e->d_abort, e->spin_limit, 0,
                                                 e->stream)
                            : launch_ensemble_x2(e->spitzer, e->saturate, e->d_probs, e->d_segs, nseg, total_items,
                                                 e->d_work, e->d_done, e->d_status, e->d_abort, e->spin_limit, 0,
                                                 e->stream);
        if (c != cudaSuccess) return efail(e, RKL_ERR_CUDA, std::string("ensemble launch: ") + cudaGetErrorString(c));
    } else {
        // one launch per problem and stage, stage-major
        for (int j = 1; j <= smax; ++j)
            for (int p = 0; p < np; ++p) {
                if (s[p] < j) continue;
                const x2::EnsProb& d = e->h_probs[p];
                StageIO io{};
                io.b = d.b;
                io.Y0 = d.T;
                io.MY0 = d.my0;
                io.coef_tab = d.coef;
                io.j = j;
                if (j == 1) {
                    io.mode = 1;
                    io.Yj = d.buf[0];
                } else {
                    io.mode = 2;
                    io.Yjm1 = d.buf[(j - 2) % 3];
                    io.Yjm2 = j == 2 ? d.T : d.buf[(j - 3) % 3];
                    io.Yj = j == s[p] ? d.T : d.buf[(j - 1) % 3];
                }
                LaunchCfg cfg{0, 3, e->spitzer ? 1 : 0, e->saturate ? 1 : 0, 0};
                KCoef<float> cf{0.f, 0.f, 0.f, 0.f};
                cudaError_t c = (e->persistent & 2)
                                    ? launch_stage_xq(cfg, d.g, d.p, io, cf, e->d_status, e->nzchunk, e->stream,
                                                      d.txw)
                                    : launch_stage_x2(cfg, d.g, d.p, io, cf, e->d_status, e->nzchunk,
                                                      d.txw == 32 ? 6 : 2, e->stream);
                if (c != cudaSuccess) return efail(e, RKL_ERR_CUDA, std::string("stage launch: ") + cudaGetErrorString(c));
            }
    }
    return RKL_OK;
}

rkl_status ens_choose_s(rkl_ensemble* e, const double* dt, std::vector<int>& s)
{
    s.assign(e->nprob, 0);
    for (int p = 0; p < e->nprob; ++p) {
        const double mx = e->h_pstats[3 * p], mn = e->h_pstats[3 * p + 1];
        if (!std::isfinite(mx) || !std::isfinite(mn)) return efail(e, RKL_ERR_NONFINITE, "T holds NaN or Inf");
        if (e->phys[p].kappa_model == RKL_KAPPA_SPITZER && !(mn > 0.0))
            return efail(e, RKL_ERR_NONPOSITIVE_T, "T must be > 0 under Spitzer kappa");
        const rkl_grid& g = e->grid[p];
        double inv = 0.0;
        for (int d = 0; d < 3; ++d) inv += 1.0 / (g.dx[d] * g.dx[d]);
        const double Tm = e->phys[p].kappa_model == RKL_KAPPA_SPITZER ? mx : 1.0;
        const double dte = e->phys[p].cp / (kpar_host(e->phys[p], Tm) * (1.0 + e->phys[p].kappa_perp_ratio) * inv);
        if (!(dt[p] > 0.0) || !std::isfinite(dt[p])) return efail(e, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
        if (rkl_num_stages(dt[p] / dte, &s[p]) != RKL_OK)
            return efail(e, RKL_ERR_INVALID_ARG, "dt/dt_expl needs more than 4096 stages");
    }
    return RKL_OK;
}

}  // namespace

extern "C" {

rkl_status rkl_ensemble_create(int nprob, const rkl_grid* grids, const rkl_phys* phys, void* cuda_stream,
                               rkl_ensemble** out)
{
    if (!out || !grids || !phys || nprob < 1 || nprob > 65536) return efail(nullptr, RKL_ERR_INVALID_ARG, "bad argument");
    *out = nullptr;
    for (int p = 0; p < nprob; ++p) {
        const rkl_grid& g = grids[p];
        const rkl_phys& ph = phys[p];
        if (g.ndim != 3 || g.dtype != RKL_F32) return efail(nullptr, RKL_ERR_UNSUPPORTED, "ensembles are 3D FP32");
        for (int d = 0; d < 3; ++d)
            if (g.n[d] < 1 || g.n[d] > 65536 || !(g.dx[d] > 0.0) || !std::isfinite(g.dx[d]))
                return efail(nullptr, RKL_ERR_INVALID_ARG, "bad n or dx");
        if (g.n[0] % 4 != 0) return efail(nullptr, RKL_ERR_UNSUPPORTED, "ensemble problems need nx % 4 == 0");
        if ((int64_t)g.n[0] * g.n[1] > ((int64_t)1 << 31)) return efail(nullptr, RKL_ERR_INVALID_ARG, "plane too large");
        if (g.bc != RKL_PERIODIC && g.bc != RKL_DIRICHLET) return efail(nullptr, RKL_ERR_INVALID_ARG, "bad bc");
        if (ph.kappa_model != phys[0].kappa_model || (ph.saturate != 0) != (phys[0].saturate != 0))
            return efail(nullptr, RKL_ERR_UNSUPPORTED, "all problems must share kappa_model and saturate");
        if (ph.kappa_model != RKL_KAPPA_CONST && ph.kappa_model != RKL_KAPPA_SPITZER)
            return efail(nullptr, RKL_ERR_INVALID_ARG, "bad kappa_model");
        if (!(ph.kappa_par0 > 0.0) || !(ph.kappa_perp_ratio >= 0.0) || !(ph.cp > 0.0 && ph.cp <= 0.5))
            return efail(nullptr, RKL_ERR_INVALID_ARG, "bad physics");
        if (ph.saturate && (!(ph.phi > 0.0) || !(ph.rho > 0.0)))
            return efail(nullptr, RKL_ERR_INVALID_ARG, "saturation needs phi > 0 and rho > 0");
        if (ph.limiter != RKL_LIMITER_NONE)
            return efail(nullptr, RKL_ERR_UNSUPPORTED, "ensembles use the arithmetic-mean transverse gradients");
    }
    rkl_ensemble* e = new rkl_ensemble();
    e->nprob = nprob;
    e->grid.assign(grids, grids + nprob);
    e->phys.assign(phys, phys + nprob);
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    e->spitzer = phys[0].kappa_model == RKL_KAPPA_SPITZER;
    e->saturate = phys[0].saturate != 0;
    e->off.assign(nprob + 1, 0);
    std::vector<int64_t> cstart;
    std::vector<int> clen, pchunk(nprob + 1, 0);
    for (int p = 0; p < nprob; ++p) {
        const rkl_grid& g = grids[p];
        const int64_t n = g.n[0] * g.n[1] * g.n[2];
        e->off[p + 1] = e->off[p] + n;                 // n % 4 == 0 since nx % 4 == 0
        KGrid<float> kg{};
        KPhys<float> kp{};
        for (int d = 0; d < 3; ++d) {
            kg.n[d] = (int)g.n[d];
            kg.inv_dx[d] = (float)(1.0 / g.dx[d]);
            kg.inv_4dx[d] = (float)(0.25 / g.dx[d]);
        }
        kg.ndim = 3;
        kg.bc = g.bc;
        kg.bcv = (float)g.bc_value;
        kg.plane = g.n[0] * g.n[1];
        kg.ncell = n;
        if (g.bc != RKL_PERIODIC || n >= ((int64_t)1 << 31)) e->rowpair_ok = false;
        kp.kappa0 = (float)phys[p].kappa_par0;
        kp.kperp = (float)phys[p].kappa_perp_ratio;
        kp.q0 = (float)(5.0 * phys[p].phi * phys[p].rho);
        kp.upwind = phys[p].sat_upwind ? 1 : 0;
        e->kg.push_back(kg);
        e->kp.push_back(kp);
        pchunk[p] = (int)cstart.size();
        for (int64_t c = 0; c < n; c += kChunk) {
            cstart.push_back(e->off[p] + c);
            clen.push_back((int)std::min<int64_t>(kChunk, n - c));
        }
    }
    pchunk[nprob] = (int)cstart.size();
    e->total = e->off[nprob];
    e->nchunk = (int)cstart.size();

    auto bail = [&](cudaError_t c, const char* w) {
        std::string m = std::string(w) + ": " + cudaGetErrorString(c);
        rkl_ensemble_destroy(e);
        return efail(nullptr, c == cudaErrorMemoryAllocation ? RKL_ERR_NOMEM : RKL_ERR_CUDA, m);
    };
    cudaError_t c;
    if ((c = cudaGetDevice(&e->device)) != cudaSuccess) return bail(c, "cudaGetDevice");
    if ((c = cudaMalloc(&e->ws, sizeof(float) * 4 * e->total)) != cudaSuccess) return bail(c, "workspace");
    if ((c = cudaMalloc(&e->d_cstart, sizeof(int64_t) * e->nchunk)) != cudaSuccess) return bail(c, "chunks");
    if ((c = cudaMalloc(&e->d_clen, sizeof(int) * e->nchunk)) != cudaSuccess) return bail(c, "chunks");
    if ((c = cudaMalloc(&e->d_pchunk, sizeof(int) * (nprob + 1))) != cudaSuccess) return bail(c, "chunks");
    if ((c = cudaMalloc(&e->d_partials, sizeof(double) * 3 * e->nchunk)) != cudaSuccess) return bail(c, "partials");
    if ((c = cudaMalloc(&e->d_pstats, sizeof(double) * 3 * nprob)) != cudaSuccess) return bail(c, "stats");
    if ((c = cudaMallocHost(&e->h_pstats, sizeof(double) * 3 * nprob)) != cudaSuccess) return bail(c, "stats");
    if ((c = cudaMalloc(&e->d_probs, sizeof(x2::EnsProb) * nprob)) != cudaSuccess) return bail(c, "probs");
    if ((c = cudaMallocHost(&e->h_probs, sizeof(x2::EnsProb) * nprob)) != cudaSuccess) return bail(c, "probs");
    if ((c = cudaMalloc(&e->d_work, sizeof(int))) != cudaSuccess) return bail(c, "work");
    if ((c = cudaMalloc(&e->d_abort, sizeof(int))) != cudaSuccess) return bail(c, "abort");
    if ((c = cudaMalloc(&e->d_done, sizeof(unsigned) * nprob)) != cudaSuccess) return bail(c, "done");
    if ((c = cudaMalloc(&e->d_status, sizeof(unsigned))) != cudaSuccess) return bail(c, "status");
    if ((c = cudaMallocHost(&e->h_status, sizeof(unsigned))) != cudaSuccess) return bail(c, "status");
    if ((c = cudaMemcpyAsync(e->d_cstart, cstart.data(), sizeof(int64_t) * e->nchunk, cudaMemcpyHostToDevice,
                             e->stream)) != cudaSuccess) return bail(c, "copy");
    if ((c = cudaMemcpyAsync(e->d_clen, clen.data(), sizeof(int) * e->nchunk, cudaMemcpyHostToDevice,
                             e->stream)) != cudaSuccess) return bail(c, "copy");
    if ((c = cudaMemcpyAsync(e->d_pchunk, pchunk.data(), sizeof(int) * (nprob + 1), cudaMemcpyHostToDevice,
                             e->stream)) != cudaSuccess) return bail(c, "copy");
    if ((c = cudaMemsetAsync(e->d_status, 0, sizeof(unsigned), e->stream)) != cudaSuccess) return bail(c, "memset");
    if ((c = cudaStreamSynchronize(e->stream)) != cudaSuccess) return bail(c, "sync");
    *out = e;
    return RKL_OK;
}

rkl_status rkl_ensemble_destroy(rkl_ensemble* e)
{
    if (!e) return RKL_ERR_INVALID_ARG;
    cudaStreamSynchronize(e->stream);
    cudaFree(e->ws);
    cudaFree(e->d_cstart);
    cudaFree(e->d_clen);
    cudaFree(e->d_pchunk);
    cudaFree(e->d_partials);
    cudaFree(e->d_pstats);
    if (e->h_pstats) cudaFreeHost(e->h_pstats);
    cudaFree(e->d_probs);
    if (e->h_probs) cudaFreeHost(e->h_probs);
    cudaFree(e->d_segs);
    if (e->h_segs) cudaFreeHost(e->h_segs);
    cudaFree(e->d_coef);
    if (e->h_coef) cudaFreeHost(e->h_coef);
    cudaFree(e->d_work);
    cudaFree(e->d_done);
    cudaFree(e->d_abort);
    cudaFree(e->d_status);
    if (e->h_status) cudaFreeHost(e->h_status);
    delete e;
    return RKL_OK;
}

const char* rkl_ensemble_last_error(const rkl_ensemble* e)
{
    return e ? e->err.c_str() : "";
}

rkl_status rkl_ensemble_layout(const rkl_ensemble* e, int64_t* cell_offsets)
{
    if (!e || !cell_offsets) return RKL_ERR_INVALID_ARG;
    for (int p = 0; p <= e->nprob; ++p) cell_offsets[p] = e->off[p];
    return RKL_OK;
}

rkl_status rkl_ensemble_set_schedule(rkl_ensemble* e, int persistent, int nzchunk)
{
    if (!e) return RKL_ERR_INVALID_ARG;
    if (nzchunk < 0 || nzchunk > 4096) return efail(e, RKL_ERR_INVALID_ARG, "nzchunk must be in [0, 4096]");
    if (persistent < 0 || persistent > 3) return efail(e, RKL_ERR_INVALID_ARG, "schedule must be 0 to 3");
    if ((persistent & 2) && !e->rowpair_ok)
        return efail(e, RKL_ERR_UNSUPPORTED, "row-pair tiles need every problem periodic with fewer than 2^31 cells");
    e->persistent = persistent;
    e->nzchunk = nzchunk > 0 ? nzchunk : 32;
    return RKL_OK;
}

rkl_status rkl_ensemble_super_step(rkl_ensemble* e, const double* dt, void* T_all, const void* b_all, int* s_used)
{
    if (!e) return RKL_ERR_INVALID_ARG;
    if (!dt || !T_all || !b_all) return efail(e, RKL_ERR_INVALID_ARG, "null argument");
    if (!al16(T_all) || !al16(b_all)) return efail(e, RKL_ERR_INVALID_ARG, "T_all and b_all must be 16-byte aligned");
    Guard gd(e->device);
    rkl_status st = ens_stats(e, static_cast<const float*>(T_all));
    if (st != RKL_OK) return st;
    std::vector<int> s;
    st = ens_choose_s(e, dt, s);
    if (st != RKL_OK) return st;
    st = ens_run(e, dt, s.data(), static_cast<float*>(T_all), static_cast<const float*>(b_all));
    if (st != RKL_OK) return st;
    e->last_s = s;
    if (s_used)
        for (int p = 0; p < e->nprob; ++p) s_used[p] = s[p];
    return RKL_OK;
}

rkl_status rkl_ensemble_check(rkl_ensemble* e)
{
    if (!e) return RKL_ERR_INVALID_ARG;
    Guard gd(e->device);
    ENS_CK(e, cudaMemcpyAsync(e->h_status, e->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_status, 0, sizeof(unsigned), e->stream));
    ENS_CK(e, cudaStreamSynchronize(e->stream));
    const unsigned w = *e->h_status;
    if (w & ST_NONFINITE) return efail(e, RKL_ERR_NONFINITE, "a stage produced NaN or Inf");
    if (w & ST_NONPOSITIVE) return efail(e, RKL_ERR_NONPOSITIVE_T, "a stage produced T <= 0 under Spitzer kappa");
    if (w & ST_TIMEOUT) return efail(e, RKL_ERR_TIMEOUT, "a bounded wait of the persistent kernel gave up");
    return RKL_OK;
}

rkl_status rkl_ensemble_autotune(rkl_ensemble* e, const double* dt, const void* T_all, const void* b_all,
                                 int* persistent_out, int* nzchunk_out, double* ms_out)
{
    if (!e) return RKL_ERR_INVALID_ARG;
    if (!dt || !T_all || !b_all) return efail(e, RKL_ERR_INVALID_ARG, "null argument");
    if (!al16(T_all) || !al16(b_all)) return efail(e, RKL_ERR_INVALID_ARG, "T_all and b_all must be 16-byte aligned");
    Guard gd(e->device);
    rkl_status st = ens_stats(e, static_cast<const float*>(T_all));
    if (st != RKL_OK) return st;
    std::vector<int> s;
    st = ens_choose_s(e, dt, s);
    if (st != RKL_OK) return st;
    float* scratch = nullptr;
    ENS_CK(e, cudaMalloc(&scratch, sizeof(float) * e->total));
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int cand[][2] = {{1, 8}, {1, 16}, {1, 32}, {3, 8}, {3, 16}, {3, 32}, {3, 48}, {3, 64},
                           {0, 16}, {0, 32}, {2, 16}, {2, 32}};
    double best = 1e300;
    int bp = 1, bz = 32;
    const int keep_p = e->persistent, keep_z = e->nzchunk;
    for (const auto& c : cand) {
        if ((c[0] & 2) && !e->rowpair_ok) continue;
        e->persistent = c[0];
        e->nzchunk = c[1];
        float ms_sum = 0.f;
        for (int rep = 0; rep < 2; ++rep) {          // first repetition warms up
            cudaMemcpyAsync(scratch, T_all, sizeof(float) * e->total, cudaMemcpyDeviceToDevice, e->stream);
            cudaEventRecord(a, e->stream);
            st = ens_run(e, dt, s.data(), scratch, static_cast<const float*>(b_all));
            cudaEventRecord(b, e->stream);
            if (st != RKL_OK) break;
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep == 1) ms_sum = ms;
        }
        if (st != RKL_OK) break;
        if (ms_sum < best) {
            best = ms_sum;
            bp = c[0];
            bz = c[1];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(e->stream);
    cudaFree(scratch);
    if (st != RKL_OK) {
        e->persistent = keep_p;
        e->nzchunk = keep_z;
        return st;
    }
    e->persistent = bp;
    e->nzchunk = bz;
    if (persistent_out) *persistent_out = bp;
    if (nzchunk_out) *nzchunk_out = bz;
    if (ms_out) *ms_out = best;
    return rkl_ensemble_check(e);
}

rkl_status rkl_ensemble_selftest_timeout(rkl_ensemble* e, int* status_out)
{
    if (!e || !status_out) return RKL_ERR_INVALID_ARG;
    Guard gd(e->device);
    // problem 0, stage 2 only: its wait for stage 1 can never be satisfied
    x2::EnsProb d{};
    d.g = e->kg[0];
    d.p = e->kp[0];
    d.nzchunk = e->nzchunk;
    set_tiles(d, e->nzchunk, false);
    d.s = 2;
    e->h_probs[0] = d;
    rkl_status st = grow_pinned(e, &e->d_segs, &e->h_segs, &e->seg_cap, 1);
    if (st != RKL_OK) return st;
    e->h_segs[0] = x2::EnsSeg{0, 0, 2, d.ntiles};
    ENS_CK(e, cudaMemcpyAsync(e->d_probs, e->h_probs, sizeof(x2::EnsProb), cudaMemcpyHostToDevice, e->stream));
    ENS_CK(e, cudaMemcpyAsync(e->d_segs, e->h_segs, sizeof(x2::EnsSeg), cudaMemcpyHostToDevice, e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_work, 0, sizeof(int), e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_abort, 0, sizeof(int), e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * e->nprob, e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_status, 0, sizeof(unsigned), e->stream));
    cudaError_t c = launch_ensemble_x2(e->spitzer, e->saturate, e->d_probs, e->d_segs, 1, d.ntiles, e->d_work,
                                       e->d_done, e->d_status, e->d_abort, 2000, 2, e->stream);
    if (c != cudaSuccess) return efail(e, RKL_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(c));
    ENS_CK(e, cudaMemcpyAsync(e->h_status, e->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
    ENS_CK(e, cudaMemsetAsync(e->d_status, 0, sizeof(unsigned), e->stream));
    ENS_CK(e, cudaStreamSynchronize(e->stream));
    *status_out = (*e->h_status & ST_TIMEOUT) ? RKL_ERR_TIMEOUT : RKL_OK;
    return RKL_OK;
}

}  // extern "C"
