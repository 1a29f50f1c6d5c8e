// C ABI of the RKL2 conduction library (see include/rkl.h): argument
// checks, the plan (workspace, coefficient table, graph cache, timing) and
// the dispatch between the tiled FP32 kernel and the generic kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rkl.h"
#include "rkl_launch.h"

using namespace rkl;

namespace {

constexpr int kMaxStages = 4096;
constexpr int kCoefRing = 8;
constexpr int kGraphCache = 16;

thread_local std::string g_create_error;

struct GraphEntry {
    int s = 0;
    const void* T = nullptr;
    const void* b = nullptr;
    int timing = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t last_use = 0;
};

}  // namespace

struct rkl_plan {
    rkl_grid grid;
    rkl_phys phys;
    cudaStream_t stream = nullptr;     // caller's stream: all work runs here
    cudaStream_t cap = nullptr;        // private stream used only to capture graphs
    int device = 0;
    size_t esize = 4;
    int64_t ncell = 0;
    LaunchCfg cfg{};
    KGrid<float> gf{};
    KGrid<double> gd{};
    KPhys<float> pf{};
    KPhys<double> pd{};
    bool fast = false;                 // tiled kernel available for this grid
    bool x2ok = false;                 // paired-cell kernel available for this grid
    int variant = 0;                   // 0 auto, 1 generic, 2 tiled, 3/4 paired-cell (2/3 CTAs per SM)
    int nzchunk = 0;                   // planes per CTA of the paired-cell kernel (0: automatic, < 0: balanced runs)

    void* ybuf[3] = {nullptr, nullptr, nullptr};
    void* ybuf4 = nullptr;             // fourth stage buffer of the two-stage kernel (allocated on use)
    bool pairok = false;               // two-stage kernel applies to the grid
    bool xqok = false;                 // row-pair kernel applies to the grid
    void* my0 = nullptr;
    double* d_partials = nullptr;
    // {max, min, sum, status} of the statistics pass, written by its last
    // block straight into page-locked mapped host memory: the read-back
    // needs no copy engine, so it never queues behind a large copy-out
    double* h_scal = nullptr;
    double* m_scal = nullptr;          // device address of h_scal
    unsigned* d_status = nullptr;

    int method = RKL_METHOD_RKL2;      // super-time-stepping method (Section 3.3)
    double sts_nu = 1e-3;              // AAG-STS damping
    void* d_coef = nullptr;            // [(kMaxStages + 1) * 4] of the grid dtype
    void* h_coef = nullptr;            // pinned [kCoefRing][(kMaxStages + 1) * 4]
    cudaEvent_t coef_ev[kCoefRing] = {};
    int coef_slot = 0;

    GraphEntry cache[kGraphCache];
    uint64_t use_clock = 0;

    int timing = 0;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    bool timing_pending = false;
    int pending_launches = 0;
    double timing_ms = 0.0;
    int64_t timing_launches = 0;

    void* host_T = nullptr;            // device staging for rkl_run_host
    void* host_b = nullptr;
    // rkl_run_host_batch: two more staging sets (three in all with host_T /
    // host_b), copy-in / copy-out streams and the events that order them
    // around the plan's stream
    void* batch_T[2] = {};
    void* batch_b[2] = {};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[3] = {}, ev_comp[3] = {}, ev_out[3] = {};

    std::string err;
};

namespace {

rkl_status fail(rkl_plan* p, rkl_status st, const std::string& msg)
{
    if (p) p->err = msg;
    else g_create_error = msg;
    return st;
}

rkl_status cuda_fail(rkl_plan* p, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(p, RKL_ERR_CUDA, m);
}

#define RKL_CK(p, call)                                                   \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail((p), e_, #call);          \
    } while (0)

bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

double kappa_par_host(const rkl_phys& ph, double T)
{
    if (ph.kappa_model == RKL_KAPPA_SPITZER) return ph.kappa_par0 * T * T * std::sqrt(T);
    return ph.kappa_par0;
}

void host_coeffs(int s, double* mu, double* nu, double* mut, double* gt)
{
    auto bj = [](int j) -> double {
        if (j <= 2) return 1.0 / 3.0;
        return ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0));
    };
    double w1 = 4.0 / ((double)s * s + s - 2.0);
    for (int j = 0; j <= s; ++j) mu[j] = nu[j] = mut[j] = gt[j] = 0.0;
    mut[1] = bj(1) * w1;
    for (int j = 2; j <= s; ++j) {
        mu[j] = (2.0 * j - 1.0) / j * bj(j) / bj(j - 1);
        nu[j] = -((double)j - 1.0) / j * bj(j) / bj(j - 2);
        mut[j] = mu[j] * w1;
        gt[j] = -(1.0 - bj(j - 1)) * mut[j];
    }
}

// Eq. AAG-STS: super-step over explicit step for N sub-steps, damping nu.
double sts_gain(int N, double nu)
{
    const double r = std::sqrt(nu);
    const double a = std::pow(1.0 + r, 2.0 * N), c = std::pow(1.0 - r, 2.0 * N);
    return N / (2.0 * r) * (a - c) / (a + c);
}

bool method_ok(int method, double nu)
{
    if (method == RKL_METHOD_RKL2 || method == RKL_METHOD_RKL1) return true;
    return method == RKL_METHOD_STS && nu > 0.0 && nu < 1.0;
}

// Stage count for dt/dt_expl = ratio (Eq. RKL-s for RKL2 and RKL1, Eq.
// AAG-STS for AAG-STS); 0 when more than kMaxStages would be needed.
int method_stages(int method, double ratio, double nu)
{
    if (method == RKL_METHOD_STS) {
        int N = 1;
        while (sts_gain(N, nu) < ratio) {
            if (++N > kMaxStages) return 0;
        }
        return N;
    }
    const double x = method == RKL_METHOD_RKL1 ? 0.5 * (-1.0 + std::sqrt(1.0 + 8.0 * ratio))
                                               : 0.5 * (-1.0 + std::sqrt(9.0 + 16.0 * ratio));
    if (x + 1.0 > (double)kMaxStages) return 0;
    return 1 + (int)std::floor(x);
}

// Coefficients of a method in the common stage form
//   Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + (1 - mu_j - nu_j) Y_0 + mut_j tau M(Y_{j-1}) + gt_j tau M(Y_0).
void method_coeffs(int method, int s, double sts_nu, double* mu, double* nu, double* mut, double* gt)
{
    if (method == RKL_METHOD_RKL2) {
        host_coeffs(s, mu, nu, mut, gt);
        return;
    }
    for (int j = 0; j <= s; ++j) mu[j] = nu[j] = mut[j] = gt[j] = 0.0;
    if (method == RKL_METHOD_RKL1) {
        const double w1 = 2.0 / ((double)s * s + s);
        mut[1] = w1;
        for (int j = 2; j <= s; ++j) {
            mu[j] = (2.0 * j - 1.0) / j;
            nu[j] = -((double)j - 1.0) / j;
            mut[j] = mu[j] * w1;
        }
        return;
    }
    // AAG-STS: sub-steps of a unit super-step (dt_p = 1 / gain(s))
    const double dtp = 1.0 / sts_gain(s, sts_nu);
    const double pi = 3.14159265358979323846;
    for (int j = 1; j <= s; ++j) {
        mu[j] = j >= 2 ? 1.0 : 0.0;
        mut[j] = dtp / ((sts_nu - 1.0) * std::cos((2.0 * j - 1.0) * pi / (2.0 * s)) + 1.0 + sts_nu);
    }
}

rkl_status check_plan(rkl_plan* p)
{
    if (!p) return RKL_ERR_INVALID_ARG;
    return RKL_OK;
}

// Launch one stage (or M) on stream st (the plan's stream, or the capture
// stream while a graph is being recorded).
rkl_status launch_stage(rkl_plan* p, const StageIO& io, double mu, double nu, double mt, double gt,
                        cudaStream_t st)
{
    cudaError_t e;
    if (p->cfg.dtype == RKL_F32) {
        KCoef<float> cf{(float)mu, (float)nu, (float)mt, (float)gt};
        bool al = aligned16(io.Y0) && aligned16(io.MY0) && aligned16(io.Yjm1) && aligned16(io.Yjm2) &&
                  aligned16(io.Yj) && aligned16(io.b);
        if ((p->variant == 0 || p->variant == 10 || p->variant == 11) && p->xqok && al) {
            // automatic choice: 32-column tiles where they leave fewer columns idle
            const int nx = (int)p->gf.n[0];
            const bool narrow = p->variant == 11 || (p->variant == 0 && (nx + 31) / 32 * 32 < (nx + 63) / 64 * 64);
            e = launch_stage_xq(p->cfg, p->gf, p->pf, io, cf, p->d_status, p->nzchunk, st, narrow ? 32 : 64);
        }
        else if (p->x2ok && al && (p->variant == 0 || (p->variant >= 3 && p->variant <= 9)))
            e = launch_stage_x2(p->cfg, p->gf, p->pf, io, cf, p->d_status, p->nzchunk,
                                p->variant == 4 ? 3 : (p->variant == 9 ? 6 : 2), st, p->variant == 6,
                                p->variant == 7, p->variant == 8);
        else if (p->fast && al && (p->variant == 0 || p->variant == 2))
            e = launch_stage_fast(p->cfg, p->gf, p->pf, io, cf, p->d_status, st);
        else
            e = launch_stage_generic(p->cfg, &p->gf, &p->pf, io, &cf, p->d_status, st);
    } else {
        KCoef<double> cf{mu, nu, mt, gt};
        e = launch_stage_generic(p->cfg, &p->gd, &p->pd, io, &cf, p->d_status, st);
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "stage launch");
    return RKL_OK;
}

// Enqueue the s stages of one super-step reading coefficients from the
// plan's device table (stage j at d_coef[4 j]).  Y0 = T; the last stage
// writes T (each cell reads its own Y0 before overwriting it).
rkl_status enqueue_stages(rkl_plan* p, int s, void* T, const void* b, bool with_events, cudaStream_t cs)
{
    StageIO io{};
    io.b = b;
    io.coef_tab = p->d_coef;
    io.Y0 = T;
    io.MY0 = p->my0;
    io.j = 1;
    io.mode = 1;
    io.Yj = p->ybuf[0];
    rkl_status st = launch_stage(p, io, 0, 0, 0, 0, cs);
    if (st != RKL_OK) return st;
    if (s == 1) {                      // single forward-Euler stage (RKL1, AAG-STS)
        RKL_CK(p, cudaMemcpyAsync(T, p->ybuf[0], (size_t)p->ncell * p->esize, cudaMemcpyDeviceToDevice, cs));
        return RKL_OK;
    }
    if (with_events) RKL_CK(p, cudaEventRecordWithFlags(p->ev_a, cs, cudaEventRecordExternal));
    if (p->variant == 5 && p->pairok && p->ybuf4) {
        // stages (j, j+1) in pairs, the last stage alone so that it may write
        // T in place; pair outputs never alias the pair's inputs (4 buffers)
        void* bufs[4] = {p->ybuf[0], p->ybuf[1], p->ybuf[2], p->ybuf4};
        const void* prev2 = T;
        void* prev1 = p->ybuf[0];
        auto pick = [&](void* avoid) {
            for (void* q : bufs)
                if (q != prev1 && q != prev2 && q != avoid) return q;
            return (void*)nullptr;
        };
        int j = 2;
        for (; j + 1 <= s - 1; j += 2) {
            StageIO q{};
            q.b = b;
            q.coef_tab = p->d_coef;
            q.Y0 = T;
            q.MY0 = p->my0;
            q.Yjm1 = prev1;
            q.Yjm2 = prev2;
            q.Yj = pick(nullptr);
            void* Yj1 = pick(q.Yj);
            q.j = j;
            q.mode = 2;
            cudaError_t e = launch_stage_pair(p->cfg, p->gf, p->pf, q, Yj1, p->d_status, p->nzchunk, cs);
            if (e != cudaSuccess) return cuda_fail(p, e, "two-stage launch");
            prev2 = q.Yj;
            prev1 = Yj1;
        }
        for (; j <= s; ++j) {
            StageIO q{};
            q.b = b;
            q.coef_tab = p->d_coef;
            q.Y0 = T;
            q.MY0 = p->my0;
            q.Yjm1 = prev1;
            q.Yjm2 = prev2;
            q.Yj = (j == s) ? T : pick(nullptr);
            q.j = j;
            q.mode = 2;
            st = launch_stage(p, q, 0, 0, 0, 0, cs);
            if (st != RKL_OK) return st;
            prev2 = prev1;
            prev1 = q.Yj;
        }
        if (with_events) RKL_CK(p, cudaEventRecordWithFlags(p->ev_b, cs, cudaEventRecordExternal));
        return RKL_OK;
    }
    for (int j = 2; j <= s; ++j) {
        StageIO q{};
        q.b = b;
        q.coef_tab = p->d_coef;
        q.Y0 = T;
        q.MY0 = p->my0;
        q.Yjm1 = p->ybuf[(j - 2) % 3];
        q.Yjm2 = (j == 2) ? T : p->ybuf[(j - 3) % 3];
        q.Yj = (j == s) ? T : p->ybuf[(j - 1) % 3];
        q.j = j;
        q.mode = 2;
        st = launch_stage(p, q, 0, 0, 0, 0, cs);
        if (st != RKL_OK) return st;
    }
    if (with_events) RKL_CK(p, cudaEventRecordWithFlags(p->ev_b, cs, cudaEventRecordExternal));
    return RKL_OK;
}

rkl_status upload_coeffs(rkl_plan* p, int s, double dt)
{
    std::vector<double> mu(s + 1), nu(s + 1), mut(s + 1), gt(s + 1);
    method_coeffs(p->method, s, p->sts_nu, mu.data(), nu.data(), mut.data(), gt.data());
    int slot = p->coef_slot;
    p->coef_slot = (p->coef_slot + 1) % kCoefRing;
    RKL_CK(p, cudaEventSynchronize(p->coef_ev[slot]));
    size_t per = (size_t)(kMaxStages + 1) * 4;
    if (p->cfg.dtype == RKL_F32) {
        float* h = static_cast<float*>(p->h_coef) + slot * per;
        for (int j = 0; j <= s; ++j) {
            h[4 * j + 0] = (float)mu[j];
            h[4 * j + 1] = (float)nu[j];
            h[4 * j + 2] = (float)(mut[j] * dt);
            h[4 * j + 3] = (float)(gt[j] * dt);
        }
        RKL_CK(p, cudaMemcpyAsync(p->d_coef, h, sizeof(float) * 4 * (s + 1), cudaMemcpyHostToDevice,
                                  p->stream));
    } else {
        double* h = static_cast<double*>(p->h_coef) + slot * per;
        for (int j = 0; j <= s; ++j) {
            h[4 * j + 0] = mu[j];
            h[4 * j + 1] = nu[j];
            h[4 * j + 2] = mut[j] * dt;
            h[4 * j + 3] = gt[j] * dt;
        }
        RKL_CK(p, cudaMemcpyAsync(p->d_coef, h, sizeof(double) * 4 * (s + 1), cudaMemcpyHostToDevice,
                                  p->stream));
    }
    RKL_CK(p, cudaEventRecord(p->coef_ev[slot], p->stream));
    return RKL_OK;
}

rkl_status get_graph(rkl_plan* p, int s, void* T, const void* b, cudaGraphExec_t* out)
{
    GraphEntry* victim = &p->cache[0];
    for (auto& g : p->cache) {
        if (g.exec && g.s == s && g.T == T && g.b == b && g.timing == p->timing) {
            g.last_use = ++p->use_clock;
            *out = g.exec;
            return RKL_OK;
        }
        if (!g.exec || g.last_use < victim->last_use) victim = &g;
    }
    if (victim->exec) {
        cudaGraphExecDestroy(victim->exec);
        victim->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    RKL_CK(p, cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    rkl_status st = enqueue_stages(p, s, T, b, p->timing != 0, p->cap);
    cudaError_t ce = cudaStreamEndCapture(p->cap, &graph);
    if (st != RKL_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess) return cuda_fail(p, ce, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(p, ce, "cudaGraphInstantiate");
    victim->s = s;
    victim->T = T;
    victim->b = b;
    victim->timing = p->timing;
    victim->exec = exec;
    victim->last_use = ++p->use_clock;
    *out = exec;
    return RKL_OK;
}

rkl_status collect_timing(rkl_plan* p)
{
    if (!p->timing_pending) return RKL_OK;
    RKL_CK(p, cudaEventSynchronize(p->ev_b));
    float ms = 0.f;
    RKL_CK(p, cudaEventElapsedTime(&ms, p->ev_a, p->ev_b));
    p->timing_ms += ms;
    p->timing_launches += p->pending_launches;
    p->timing_pending = false;
    return RKL_OK;
}

// FP64 {max, min, sum, status} of a device array into p->h_scal
// (synchronises).  With take_status the device status word is read into
// h_scal[3] and cleared; otherwise h_scal[3] = 0 and the word is kept.
rkl_status stats(rkl_plan* p, const void* T, bool take_status = true, bool need_sum = true)
{
    cudaError_t e = launch_stats(p->cfg.dtype, T, p->ncell, p->d_partials, p->m_scal,
                                 take_status ? p->d_status : nullptr, p->stream, need_sum);
    if (e != cudaSuccess) return cuda_fail(p, e, "stats launch");
    RKL_CK(p, cudaStreamSynchronize(p->stream));
    return RKL_OK;
}

rkl_status status_from_word(rkl_plan* p, unsigned w)
{
    if (w & ST_NONFINITE) return fail(p, RKL_ERR_NONFINITE, "a stage produced NaN or Inf");
    if (w & ST_NONPOSITIVE) return fail(p, RKL_ERR_NONPOSITIVE_T, "a stage produced T <= 0 under Spitzer kappa");
    if (w & ST_TIMEOUT) return fail(p, RKL_ERR_TIMEOUT, "a bounded device wait gave up");
    return RKL_OK;
}

double cell_volume(const rkl_grid& g)
{
    double v = 1.0;
    for (int d = 0; d < g.ndim; ++d) v *= g.dx[d];
    return v;
}

double dt_expl_from_max(const rkl_plan* p, double Tmax)
{
    double inv = 0.0;
    for (int d = 0; d < p->grid.ndim; ++d) inv += 1.0 / (p->grid.dx[d] * p->grid.dx[d]);
    double chi = kappa_par_host(p->phys, Tmax) * (1.0 + p->phys.kappa_perp_ratio);
    return p->phys.cp / (chi * inv);
}

rkl_status run_super_step(rkl_plan* p, double dt, int s, void* T, const void* b, double* eb, double* ea)
{
    rkl_status st = upload_coeffs(p, s, dt);
    if (st != RKL_OK) return st;
    cudaGraphExec_t exec = nullptr;
    st = get_graph(p, s, T, b, &exec);
    if (st != RKL_OK) return st;
    RKL_CK(p, cudaGraphLaunch(exec, p->stream));
    if (p->timing && s >= 2) {         // events bracket stages 2..s
        p->timing_pending = true;
        p->pending_launches = s - 1;
    }
    if (ea) {
        st = stats(p, T);
        if (st != RKL_OK) return st;
        *ea = p->h_scal[2] * cell_volume(p->grid);
        st = status_from_word(p, (unsigned)p->h_scal[3]);
        if (st != RKL_OK) return st;
    }
    (void)eb;
    return RKL_OK;
}

}  // namespace

namespace rkl {
// Message for entry points without a plan (read back by rkl_last_error(NULL)).
void set_unplanned_error(const std::string& msg) { g_create_error = msg; }
// Read-only views of a plan for other parts of the library.
const rkl_grid* plan_grid(const rkl_plan* p) { return &p->grid; }
const rkl_phys* plan_phys(const rkl_plan* p) { return &p->phys; }
cudaStream_t plan_stream(const rkl_plan* p) { return p->stream; }
}  // namespace rkl

extern "C" {

const char* rkl_status_string(rkl_status st)
{
    switch (st) {
        case RKL_OK: return "RKL_OK";
        case RKL_ERR_INVALID_ARG: return "RKL_ERR_INVALID_ARG";
        case RKL_ERR_CUDA: return "RKL_ERR_CUDA";
        case RKL_ERR_NONFINITE: return "RKL_ERR_NONFINITE";
        case RKL_ERR_NONPOSITIVE_T: return "RKL_ERR_NONPOSITIVE_T";
        case RKL_ERR_TIMEOUT: return "RKL_ERR_TIMEOUT";
        case RKL_ERR_UNSUPPORTED: return "RKL_ERR_UNSUPPORTED";
        case RKL_ERR_NOMEM: return "RKL_ERR_NOMEM";
    }
    return "RKL_ERR_UNKNOWN";
}

const char* rkl_last_error(const rkl_plan* plan)
{
    if (!plan) return g_create_error.c_str();
    return plan->err.c_str();
}

rkl_status rkl_num_stages(double ratio, int* s_out)
{
    if (!s_out || !std::isfinite(ratio) || ratio <= 0.0) return RKL_ERR_INVALID_ARG;
    double s = 0.5 * (-1.0 + std::sqrt(9.0 + 16.0 * ratio));
    if (s + 1.0 > (double)kMaxStages) return RKL_ERR_INVALID_ARG;
    *s_out = 1 + (int)std::floor(s);
    return RKL_OK;
}

rkl_status rkl_coeffs(int s, double* mu, double* nu, double* mut, double* gt)
{
    if (s < 2 || s > kMaxStages || !mu || !nu || !mut || !gt) return RKL_ERR_INVALID_ARG;
    host_coeffs(s, mu, nu, mut, gt);
    return RKL_OK;
}

rkl_status rkl_num_stages_method(int method, double ratio, double sts_nu, int* s_out)
{
    if (!s_out || !std::isfinite(ratio) || ratio <= 0.0 || !method_ok(method, sts_nu)) return RKL_ERR_INVALID_ARG;
    const int s = method_stages(method, ratio, sts_nu);
    if (s == 0) return RKL_ERR_INVALID_ARG;
    *s_out = s;
    return RKL_OK;
}

rkl_status rkl_coeffs_method(int method, int s, double sts_nu, double* mu, double* nu, double* mut, double* gt)
{
    if (!method_ok(method, sts_nu) || !mu || !nu || !mut || !gt) return RKL_ERR_INVALID_ARG;
    if (s < (method == RKL_METHOD_RKL2 ? 2 : 1) || s > kMaxStages) return RKL_ERR_INVALID_ARG;
    method_coeffs(method, s, sts_nu, mu, nu, mut, gt);
    return RKL_OK;
}

rkl_status rkl_plan_set_method(rkl_plan* p, int method, double sts_nu)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!method_ok(method, sts_nu)) return fail(p, RKL_ERR_INVALID_ARG, "unknown method or sts_nu outside (0, 1)");
    p->method = method;
    if (method == RKL_METHOD_STS) p->sts_nu = sts_nu;
    return RKL_OK;
}

rkl_status rkl_plan_create(const rkl_grid* grid, const rkl_phys* phys, void* cuda_stream, rkl_plan** out)
{
    if (!grid || !phys || !out) return fail(nullptr, RKL_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    const rkl_grid& g = *grid;
    if (g.ndim < 1 || g.ndim > 3) return fail(nullptr, RKL_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        if (g.n[d] < 1 || g.n[d] > (1 << 20)) return fail(nullptr, RKL_ERR_INVALID_ARG, "bad n");
        if (d >= g.ndim && g.n[d] != 1) return fail(nullptr, RKL_ERR_INVALID_ARG, "inactive axis must have n = 1");
        if (d < g.ndim && !(g.dx[d] > 0.0 && std::isfinite(g.dx[d])))
            return fail(nullptr, RKL_ERR_INVALID_ARG, "dx must be finite and > 0");
        ncell *= g.n[d];
    }
    if (ncell > ((int64_t)1 << 34)) return fail(nullptr, RKL_ERR_INVALID_ARG, "grid too large");
    if (g.bc != RKL_PERIODIC && g.bc != RKL_DIRICHLET) return fail(nullptr, RKL_ERR_INVALID_ARG, "bad bc");
    if (g.dtype != RKL_F32 && g.dtype != RKL_F64) return fail(nullptr, RKL_ERR_INVALID_ARG, "bad dtype");
    const rkl_phys& ph = *phys;
    if (ph.kappa_model != RKL_KAPPA_CONST && ph.kappa_model != RKL_KAPPA_SPITZER)
        return fail(nullptr, RKL_ERR_INVALID_ARG, "bad kappa_model");
    if (!(ph.kappa_par0 > 0.0) || !std::isfinite(ph.kappa_par0) || !(ph.kappa_perp_ratio >= 0.0) ||
        !std::isfinite(ph.kappa_perp_ratio))
        return fail(nullptr, RKL_ERR_INVALID_ARG, "bad conductivity");
    if (!(ph.cp > 0.0 && ph.cp <= 0.5)) return fail(nullptr, RKL_ERR_INVALID_ARG, "cp must be in (0, 1/2]");
    if (ph.saturate && (!(ph.phi > 0.0) || !(ph.rho > 0.0)))
        return fail(nullptr, RKL_ERR_INVALID_ARG, "saturation needs phi > 0 and rho > 0");
    if ((ph.limiter != RKL_LIMITER_NONE && ph.limiter != RKL_LIMITER_MC) || std::isnan(ph.limiter_floor))
        return fail(nullptr, RKL_ERR_INVALID_ARG, "limiter must be RKL_LIMITER_NONE or RKL_LIMITER_MC with a floor");

    rkl_plan* p = new rkl_plan();
    p->grid = g;
    p->phys = ph;
    p->stream = static_cast<cudaStream_t>(cuda_stream);
    p->esize = g.dtype == RKL_F64 ? 8 : 4;
    p->ncell = ncell;
    p->cfg = LaunchCfg{g.dtype, g.ndim, ph.kappa_model == RKL_KAPPA_SPITZER, ph.saturate != 0,
                       ph.limiter == RKL_LIMITER_MC,
                       ph.limiter == RKL_LIMITER_MC && std::isinf(ph.limiter_floor) && ph.limiter_floor > 0};
    auto fill = [&](auto& kg, auto& kp) {
        using R = std::remove_reference_t<decltype(kg.bcv)>;
        for (int d = 0; d < 3; ++d) {
            kg.n[d] = (int)g.n[d];
            kg.inv_dx[d] = d < g.ndim ? (R)(1.0 / g.dx[d]) : R(0);
            kg.inv_4dx[d] = d < g.ndim ? (R)(0.25 / g.dx[d]) : R(0);
        }
        kg.ndim = g.ndim;
        kg.bc = g.bc;
        kg.bcv = (R)g.bc_value;
        kg.plane = g.n[0] * g.n[1];
        kg.ncell = ncell;
        kp.kappa0 = (R)ph.kappa_par0;
        kp.kperp = (R)ph.kappa_perp_ratio;
        kp.q0 = (R)(5.0 * ph.phi * ph.rho);
        kp.upwind = ph.sat_upwind ? 1 : 0;
        kp.limiter = ph.limiter == RKL_LIMITER_MC ? 1 : 0;
        kp.lfloor = std::isinf(ph.limiter_floor) ? (ph.limiter_floor > 0 ? (R)INFINITY : (R)-INFINITY)
                                                 : (R)ph.limiter_floor;
    };
    fill(p->gf, p->pf);
    fill(p->gd, p->pd);
    p->fast = g.dtype == RKL_F32 && fast_stage_supported(p->cfg, p->gf);
    p->x2ok = g.dtype == RKL_F32 && x2_stage_supported(p->cfg, p->gf);
    p->pairok = g.dtype == RKL_F32 && pair_stage_supported(p->cfg, p->gf);
    p->xqok = g.dtype == RKL_F32 && xq_stage_supported(p->cfg, p->gf);

    rkl_plan* P = p;
    auto bail = [&](cudaError_t e, const char* where) {
        std::string m = std::string(where) + ": " + cudaGetErrorString(e);
        rkl_plan_destroy(P);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? RKL_ERR_NOMEM : RKL_ERR_CUDA, m);
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&p->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
    if ((e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(e, "cudaStreamCreate");
    size_t bytes = (size_t)ncell * p->esize;
    for (int k = 0; k < 3; ++k)
        if ((e = cudaMalloc(&p->ybuf[k], bytes)) != cudaSuccess) return bail(e, "cudaMalloc(stage buffer)");
    if ((e = cudaMalloc(&p->my0, bytes)) != cudaSuccess) return bail(e, "cudaMalloc(MY0)");
    // partials of the statistics pass, then its block ticket counter (zeroed)
    if ((e = cudaMalloc(&p->d_partials, sizeof(double) * (3 * kStatsBlocks + 1))) != cudaSuccess)
        return bail(e, "cudaMalloc(partials)");
    if ((e = cudaMemsetAsync(p->d_partials, 0, sizeof(double) * (3 * kStatsBlocks + 1), p->stream)) != cudaSuccess)
        return bail(e, "cudaMemset(partials)");
    if ((e = cudaHostAlloc(&p->h_scal, sizeof(double) * 4, cudaHostAllocMapped)) != cudaSuccess)
        return bail(e, "cudaHostAlloc(scalars)");
    if ((e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&p->m_scal), p->h_scal, 0)) != cudaSuccess)
        return bail(e, "cudaHostGetDevicePointer(scalars)");
    if ((e = cudaMalloc(&p->d_status, sizeof(unsigned))) != cudaSuccess) return bail(e, "cudaMalloc(status)");
    if ((e = cudaMemsetAsync(p->d_status, 0, sizeof(unsigned), p->stream)) != cudaSuccess)
        return bail(e, "cudaMemset(status)");
    size_t per = (size_t)(kMaxStages + 1) * 4 * p->esize;
    if ((e = cudaMalloc(&p->d_coef, per)) != cudaSuccess) return bail(e, "cudaMalloc(coef)");
    if ((e = cudaMallocHost(&p->h_coef, per * kCoefRing)) != cudaSuccess) return bail(e, "cudaMallocHost(coef)");
    for (int k = 0; k < kCoefRing; ++k)
        if ((e = cudaEventCreateWithFlags(&p->coef_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&p->ev_a)) != cudaSuccess) return bail(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&p->ev_b)) != cudaSuccess) return bail(e, "cudaEventCreate");
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return bail(e, "cudaStreamSynchronize");
    *out = p;
    return RKL_OK;
}

rkl_status rkl_plan_destroy(rkl_plan* p)
{
    if (!p) return RKL_ERR_INVALID_ARG;
    cudaStreamSynchronize(p->stream);
    for (auto& g : p->cache)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < 3; ++k) cudaFree(p->ybuf[k]);
    cudaFree(p->ybuf4);
    cudaFree(p->my0);
    if (p->s_in) cudaStreamSynchronize(p->s_in);
    if (p->s_out) cudaStreamSynchronize(p->s_out);
    for (int k = 0; k < 2; ++k) {
        cudaFree(p->batch_T[k]);
        cudaFree(p->batch_b[k]);
    }
    for (int k = 0; k < 3; ++k) {
        if (p->ev_in[k]) cudaEventDestroy(p->ev_in[k]);
        if (p->ev_comp[k]) cudaEventDestroy(p->ev_comp[k]);
        if (p->ev_out[k]) cudaEventDestroy(p->ev_out[k]);
    }
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    cudaFree(p->d_partials);
    if (p->h_scal) cudaFreeHost(p->h_scal);
    cudaFree(p->d_status);
    cudaFree(p->d_coef);
    if (p->h_coef) cudaFreeHost(p->h_coef);
    for (int k = 0; k < kCoefRing; ++k)
        if (p->coef_ev[k]) cudaEventDestroy(p->coef_ev[k]);
    if (p->ev_a) cudaEventDestroy(p->ev_a);
    if (p->ev_b) cudaEventDestroy(p->ev_b);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaFree(p->host_T);
    cudaFree(p->host_b);
    delete p;
    return RKL_OK;
}

rkl_status rkl_dt_expl(rkl_plan* p, const void* T, double* dt_out)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!T || !dt_out) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    DeviceGuard dg(p->device);
    double Tmax = 1.0;
    if (p->phys.kappa_model == RKL_KAPPA_SPITZER) {
        rkl_status st = stats(p, T, true, false);
        if (st != RKL_OK) return st;
        Tmax = p->h_scal[0];
        if (!(p->h_scal[1] > 0.0) || !std::isfinite(Tmax))
            return fail(p, RKL_ERR_NONPOSITIVE_T, "T must be finite and > 0 under Spitzer kappa");
    }
    *dt_out = dt_expl_from_max(p, Tmax);
    return RKL_OK;
}

rkl_status rkl_flux(rkl_plan* p, const void* T, const void* b, void* Fx, void* Fy, void* Fz)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    void* F[3] = {Fx, Fy, Fz};
    if (!T || !b) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    for (int d = 0; d < p->grid.ndim; ++d)
        if (!F[d]) return fail(p, RKL_ERR_INVALID_ARG, "missing face array");
    DeviceGuard dg(p->device);
    const void* grid = p->cfg.dtype == RKL_F32 ? (const void*)&p->gf : (const void*)&p->gd;
    const void* phys = p->cfg.dtype == RKL_F32 ? (const void*)&p->pf : (const void*)&p->pd;
    cudaError_t e = launch_flux_generic(p->cfg, grid, phys, T, b, F, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "flux launch");
    return RKL_OK;
}

rkl_status rkl_apply_M(rkl_plan* p, const void* T, const void* b, void* MT)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!T || !b || !MT) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (MT == T) return fail(p, RKL_ERR_INVALID_ARG, "MT must not alias T");
    DeviceGuard dg(p->device);
    StageIO io{};
    io.Yjm1 = T;
    io.Y0 = T;
    io.Yj = MT;
    io.b = b;
    io.mode = 0;
    return launch_stage(p, io, 0, 0, 0, 0, p->stream);
}

rkl_status rkl_stage(rkl_plan* p, int j, int s, double dt, const void* b, const void* Y0, void* MY0,
                     const void* Yjm1, const void* Yjm2, void* Yj)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (s < 1 || s > kMaxStages || j < 1 || j > s) return fail(p, RKL_ERR_INVALID_ARG, "need 1 <= j <= s <= 4096");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!b || !Y0 || !Yj) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (j >= 2 && (!MY0 || !Yjm1 || !Yjm2)) return fail(p, RKL_ERR_INVALID_ARG, "stage j >= 2 needs MY0, Yjm1, Yjm2");
    if (j == 1 && s >= 2 && !MY0) return fail(p, RKL_ERR_INVALID_ARG, "stage 1 needs MY0");
    if (j >= 2 && (Yj == Yjm1 || Yj == Yjm2 || Yj == MY0)) return fail(p, RKL_ERR_INVALID_ARG, "Yj aliases an input");
    if (j == 1 && (Yj == MY0 || Yj == Y0)) return fail(p, RKL_ERR_INVALID_ARG, "stage 1 output aliases an input");
    DeviceGuard dg(p->device);
    StageIO io{};
    io.b = b;
    io.Y0 = Y0;
    io.MY0 = MY0;
    io.Yjm1 = Yjm1;
    io.Yjm2 = Yjm2;
    io.Yj = Yj;
    io.j = j;
    if (s == 1) {
        io.mode = 1;
        io.MY0 = nullptr;
        return launch_stage(p, io, 0, 0, dt, 0, p->stream);
    }
    std::vector<double> mu(s + 1), nu(s + 1), mut(s + 1), gt(s + 1);
    method_coeffs(p->method, s, p->sts_nu, mu.data(), nu.data(), mut.data(), gt.data());
    io.mode = j == 1 ? 1 : 2;
    return launch_stage(p, io, mu[j], nu[j], mut[j] * dt, gt[j] * dt, p->stream);
}

rkl_status rkl_super_step(rkl_plan* p, double dt, void* T, const void* b, int* s_used, double* eb, double* ea)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!T || !b) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (!aligned16(T) || !aligned16(b)) return fail(p, RKL_ERR_INVALID_ARG, "T and b must be 16-byte aligned");
    DeviceGuard dg(p->device);
    rkl_status st = collect_timing(p);
    if (st != RKL_OK) return st;
    double Tmax = 1.0;
    bool need_stats = p->phys.kappa_model == RKL_KAPPA_SPITZER || eb != nullptr;
    if (need_stats) {
        st = stats(p, T, true, eb != nullptr);
        if (st != RKL_OK) return st;
        st = status_from_word(p, (unsigned)p->h_scal[3]);
        if (st != RKL_OK) return st;
        Tmax = p->h_scal[0];
        if (!std::isfinite(p->h_scal[0]) || !std::isfinite(p->h_scal[1]))
            return fail(p, RKL_ERR_NONFINITE, "T holds NaN or Inf");
        if (p->phys.kappa_model == RKL_KAPPA_SPITZER && !(p->h_scal[1] > 0.0))
            return fail(p, RKL_ERR_NONPOSITIVE_T, "T must be > 0 under Spitzer kappa");
        if (eb) *eb = p->h_scal[2] * cell_volume(p->grid);
    }
    double dte = dt_expl_from_max(p, Tmax);
    const int s = method_stages(p->method, dt / dte, p->sts_nu);
    if (s == 0) return fail(p, RKL_ERR_INVALID_ARG, "dt/dt_expl needs more than 4096 stages");
    if (s_used) *s_used = s;
    return run_super_step(p, dt, s, T, b, nullptr, ea);
}

rkl_status rkl_super_step_s(rkl_plan* p, double dt, int s, void* T, const void* b, double* eb, double* ea)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
    const int smin = p->method == RKL_METHOD_RKL2 ? 2 : 1;
    if (s < smin || s > kMaxStages) return fail(p, RKL_ERR_INVALID_ARG, "need 2 <= s <= 4096 (1 <= s for RKL1, AAG-STS)");
    if (!T || !b) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (!aligned16(T) || !aligned16(b)) return fail(p, RKL_ERR_INVALID_ARG, "T and b must be 16-byte aligned");
    DeviceGuard dg(p->device);
    rkl_status st = collect_timing(p);
    if (st != RKL_OK) return st;
    if (eb) {
        st = stats(p, T);
        if (st != RKL_OK) return st;
        *eb = p->h_scal[2] * cell_volume(p->grid);
        st = status_from_word(p, (unsigned)p->h_scal[3]);
        if (st != RKL_OK) return st;
    }
    return run_super_step(p, dt, s, T, b, nullptr, ea);
}

rkl_status rkl_energy(rkl_plan* p, const void* T, double* E_out)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!T || !E_out) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    DeviceGuard dg(p->device);
    // leaves the device status word untouched
    rkl_status st = stats(p, T, false);
    if (st != RKL_OK) return st;
    *E_out = p->h_scal[2] * cell_volume(p->grid);
    return RKL_OK;
}

rkl_status rkl_dt_hyperbolic(rkl_plan* p, const void* u, double ch, double* dt_out)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!u || !dt_out) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (!(ch > 0.0) || !std::isfinite(ch)) return fail(p, RKL_ERR_INVALID_ARG, "C_h must be finite and > 0");
    DeviceGuard dg(p->device);
    // the rates go to a stage buffer, free between super-steps
    cudaError_t e = launch_hyp_rate(p->cfg, p->cfg.dtype == RKL_F64 ? (const void*)&p->gd : (const void*)&p->gf, u,
                                    p->ybuf[0], p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "rate launch");
    rkl_status st = stats(p, p->ybuf[0], false, false);
    if (st != RKL_OK) return st;
    const double mx = p->h_scal[0];
    if (!std::isfinite(mx)) return fail(p, RKL_ERR_NONFINITE, "u holds NaN or Inf");
    *dt_out = mx > 0.0 ? ch / mx : 0.0;
    return RKL_OK;
}

rkl_status rkl_advect(rkl_plan* p, double dt, const void* u, const void* T_in, void* T_out)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!u || !T_in || !T_out) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (T_out == T_in) return fail(p, RKL_ERR_INVALID_ARG, "T_out aliases T_in");
    if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and >= 0");
    DeviceGuard dg(p->device);
    cudaError_t e = launch_advect(p->cfg, p->cfg.dtype == RKL_F64 ? (const void*)&p->gd : (const void*)&p->gf, T_in,
                                  u, T_out, dt, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "advect launch");
    return RKL_OK;
}

rkl_status rkl_plan_autotune(rkl_plan* p, double dt, const void* T, const void* b, int* variant_out,
                             int* nzchunk_out, double* ms_out)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!T || !b) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!aligned16(T) || !aligned16(b)) return fail(p, RKL_ERR_INVALID_ARG, "T and b must be 16-byte aligned");
    DeviceGuard dg(p->device);
    double dte = 0.0;
    rkl_status st = rkl_dt_expl(p, T, &dte);
    if (st != RKL_OK) return st;
    const int s = method_stages(p->method, dt / dte, p->sts_nu);
    if (s == 0) return fail(p, RKL_ERR_INVALID_ARG, "dt/dt_expl too large");
    struct Cand { int v, nz; };
    std::vector<Cand> cands = {{1, 0}};
    if (p->fast) cands.push_back({2, 0});
    // a limiter plan has one paired-cell build (variants 3-7 all launch it)
    const bool lim = p->cfg.limiter != 0;
    if (p->x2ok)
        for (int nz : {0, -1, 16, 32, 64}) {
            cands.push_back({3, nz});
            if (!lim) cands.push_back({4, nz});
            if (!lim) cands.push_back({9, nz});
        }
    if (p->x2ok && p->pairok)
        for (int nz : {16, 32, 64}) cands.push_back({5, nz});
    if (p->x2ok && !lim && p->gf.bc == 0 && p->gf.n[0] >= 72)
        for (int nz : {0, 32}) cands.push_back({6, nz});
    if (p->x2ok && !lim && x2_ytma_supported(p->cfg, p->gf)) cands.push_back({7, 0});
    if (p->x2ok && x2_tmaps_supported(p->cfg, p->gf))
        for (int nz : {0, -1, 32}) cands.push_back({8, nz});
    if (p->xqok)
        for (int nz : {0, 16, 32}) {
            cands.push_back({10, nz});
            cands.push_back({11, nz});
        }
    void* scratch = nullptr;
    RKL_CK(p, cudaMalloc(&scratch, (size_t)p->ncell * p->esize));
    cudaEvent_t a = nullptr, e = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&e);
    const int keep_v = p->variant, keep_nz = p->nzchunk;
    double best = 1e300;
    Cand bc = cands[0];
    for (const Cand& c : cands) {
        if (rkl_plan_set_variant(p, c.v, c.nz) != RKL_OK) continue;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == RKL_OK; ++rep) {          // the first repetition warms up
            cudaMemcpyAsync(scratch, T, (size_t)p->ncell * p->esize, cudaMemcpyDeviceToDevice, p->stream);
            cudaEventRecord(a, p->stream);
            st = rkl_super_step_s(p, dt, s, scratch, b, nullptr, nullptr);
            cudaEventRecord(e, p->stream);
            cudaEventSynchronize(e);
            cudaEventElapsedTime(&ms, a, e);
        }
        if (st != RKL_OK) break;
        if (ms < best) {
            best = ms;
            bc = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    cudaFree(scratch);
    if (st != RKL_OK) {
        rkl_plan_set_variant(p, keep_v, keep_nz);
        return st;
    }
    rkl_plan_set_variant(p, bc.v, bc.nz);
    if (variant_out) *variant_out = bc.v;
    if (nzchunk_out) *nzchunk_out = p->nzchunk;
    if (ms_out) *ms_out = best;
    return rkl_plan_check(p);
}

rkl_status rkl_plan_set_variant(rkl_plan* p, int variant, int nzchunk)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (variant < 0 || variant > 11) return fail(p, RKL_ERR_INVALID_ARG, "variant must be 0 to 11");
    if (nzchunk > 4096) return fail(p, RKL_ERR_INVALID_ARG, "nzchunk must be <= 4096");
    if (variant == 2 && !p->fast) return fail(p, RKL_ERR_UNSUPPORTED, "no tiled kernel for this grid");
    if ((variant == 3 || variant == 4 || (variant >= 6 && variant <= 9)) && !p->x2ok)
        return fail(p, RKL_ERR_UNSUPPORTED, "no paired-cell kernel for this grid");
    if ((variant == 10 || variant == 11) && !p->xqok)
        return fail(p, RKL_ERR_UNSUPPORTED,
                    "no row-pair kernel for this grid (periodic FP32 3D, nx % 4 == 0, no limiter or the limiter at every face, < 2^31 cells)");
    if (variant == 5 && !(p->pairok && p->x2ok))
        return fail(p, RKL_ERR_UNSUPPORTED, "no two-stage kernel for this grid (periodic FP32 3D, nx % 4 == 0)");
    if (variant == 5 && !p->ybuf4) {
        DeviceGuard dg(p->device);
        if (cudaMalloc(&p->ybuf4, (size_t)p->ncell * p->esize) != cudaSuccess) {
            cudaGetLastError();
            return fail(p, RKL_ERR_NOMEM, "cudaMalloc(fourth stage buffer)");
        }
    }
    p->nzchunk = nzchunk;
    DeviceGuard dg(p->device);
    cudaStreamSynchronize(p->stream);
    for (auto& g : p->cache)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
    p->variant = variant;
    return RKL_OK;
}

rkl_status rkl_plan_check(rkl_plan* p)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    unsigned w = 0;
    RKL_CK(p, cudaMemcpyAsync(&w, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream));
    RKL_CK(p, cudaMemsetAsync(p->d_status, 0, sizeof(unsigned), p->stream));
    RKL_CK(p, cudaStreamSynchronize(p->stream));
    return status_from_word(p, w);
}

rkl_status rkl_plan_set_timing(rkl_plan* p, int on)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    DeviceGuard dg(p->device);
    rkl_status st = collect_timing(p);
    if (st != RKL_OK) return st;
    p->timing = on ? 1 : 0;
    p->timing_ms = 0.0;
    p->timing_launches = 0;
    return RKL_OK;
}

rkl_status rkl_plan_timing(rkl_plan* p, double* ms_total, int64_t* launches)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!ms_total || !launches) return fail(p, RKL_ERR_INVALID_ARG, "null argument");
    DeviceGuard dg(p->device);
    rkl_status st = collect_timing(p);
    if (st != RKL_OK) return st;
    *ms_total = p->timing_ms;
    *launches = p->timing_launches;
    return RKL_OK;
}

rkl_status rkl_run_host(rkl_plan* p, double dt, int n_super, void* T_host, const void* b_host, int* s_last)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!T_host || !b_host || n_super < 0) return fail(p, RKL_ERR_INVALID_ARG, "bad argument");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
    DeviceGuard dg(p->device);
    size_t bytes = (size_t)p->ncell * p->esize;
    if (!p->host_T) RKL_CK(p, cudaMalloc(&p->host_T, bytes));
    if (!p->host_b) RKL_CK(p, cudaMalloc(&p->host_b, bytes * p->grid.ndim));
    RKL_CK(p, cudaMemcpyAsync(p->host_T, T_host, bytes, cudaMemcpyHostToDevice, p->stream));
    RKL_CK(p, cudaMemcpyAsync(p->host_b, b_host, bytes * p->grid.ndim, cudaMemcpyHostToDevice, p->stream));
    int s = 0;
    for (int k = 0; k < n_super; ++k) {
        rkl_status st = rkl_super_step(p, dt, p->host_T, p->host_b, &s, nullptr, nullptr);
        if (st != RKL_OK) return st;
    }
    RKL_CK(p, cudaMemcpyAsync(T_host, p->host_T, bytes, cudaMemcpyDeviceToHost, p->stream));
    RKL_CK(p, cudaStreamSynchronize(p->stream));
    if (s_last) *s_last = s;
    return rkl_plan_check(p);
}

rkl_status rkl_run_host_batch(rkl_plan* p, double dt, int n_super, int n_jobs, void* const* T_host,
                              const void* const* b_host, int* s_last)
{
    if (check_plan(p) != RKL_OK) return RKL_ERR_INVALID_ARG;
    if (!T_host || !b_host || n_super < 0 || n_jobs < 0) return fail(p, RKL_ERR_INVALID_ARG, "bad argument");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, RKL_ERR_INVALID_ARG, "dt must be finite and > 0");
    for (int i = 0; i < n_jobs; ++i)
        if (!T_host[i] || !b_host[i]) return fail(p, RKL_ERR_INVALID_ARG, "null host buffer");
    DeviceGuard dg(p->device);
    const size_t bytes = (size_t)p->ncell * p->esize, bbytes = bytes * p->grid.ndim;
    if (!p->host_T) RKL_CK(p, cudaMalloc(&p->host_T, bytes));
    if (!p->host_b) RKL_CK(p, cudaMalloc(&p->host_b, bbytes));
    for (int k = 0; k < 2; ++k) {
        if (!p->batch_T[k]) RKL_CK(p, cudaMalloc(&p->batch_T[k], bytes));
        if (!p->batch_b[k]) RKL_CK(p, cudaMalloc(&p->batch_b[k], bbytes));
    }
    if (!p->s_in) RKL_CK(p, cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking));
    if (!p->s_out) RKL_CK(p, cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking));
    for (int k = 0; k < 3; ++k) {
        if (!p->ev_in[k]) RKL_CK(p, cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming));
        if (!p->ev_comp[k]) RKL_CK(p, cudaEventCreateWithFlags(&p->ev_comp[k], cudaEventDisableTiming));
        if (!p->ev_out[k]) RKL_CK(p, cudaEventCreateWithFlags(&p->ev_out[k], cudaEventDisableTiming));
    }
    void* dT[3] = {p->host_T, p->batch_T[0], p->batch_T[1]};
    void* db[3] = {p->host_b, p->batch_b[0], p->batch_b[1]};
    // work already queued on the plan's stream may still use the staging set
    RKL_CK(p, cudaEventRecord(p->ev_comp[0], p->stream));
    RKL_CK(p, cudaStreamWaitEvent(p->s_in, p->ev_comp[0], 0));
    for (int i = 0; i < n_jobs; ++i) {
        const int k = i % 3;
        // copy-in of job i after the copy-out of job i - 3, which used the same
        // set, and after that of job i - 2 if it returns into the same host
        // buffer job i reads (the copy-in and copy-out streams otherwise run
        // side by side)
        if (i >= 3) RKL_CK(p, cudaStreamWaitEvent(p->s_in, p->ev_out[k], 0));
        if (i >= 2 && T_host[i] == T_host[i - 2])
            RKL_CK(p, cudaStreamWaitEvent(p->s_in, p->ev_out[(i - 2) % 3], 0));
        RKL_CK(p, cudaMemcpyAsync(dT[k], T_host[i], bytes, cudaMemcpyHostToDevice, p->s_in));
        RKL_CK(p, cudaMemcpyAsync(db[k], b_host[i], bbytes, cudaMemcpyHostToDevice, p->s_in));
        RKL_CK(p, cudaEventRecord(p->ev_in[k], p->s_in));
        RKL_CK(p, cudaStreamWaitEvent(p->stream, p->ev_in[k], 0));
        int s = 0;
        for (int n = 0; n < n_super; ++n) {
            rkl_status st = rkl_super_step(p, dt, dT[k], db[k], &s, nullptr, nullptr);
            if (st != RKL_OK) {
                cudaStreamSynchronize(p->s_in);
                cudaStreamSynchronize(p->s_out);
                return st;
            }
        }
        RKL_CK(p, cudaEventRecord(p->ev_comp[k], p->stream));
        RKL_CK(p, cudaStreamWaitEvent(p->s_out, p->ev_comp[k], 0));
        RKL_CK(p, cudaMemcpyAsync(T_host[i], dT[k], bytes, cudaMemcpyDeviceToHost, p->s_out));
        RKL_CK(p, cudaEventRecord(p->ev_out[k], p->s_out));
        if (s_last) s_last[i] = s;
    }
    RKL_CK(p, cudaStreamSynchronize(p->s_out));
    RKL_CK(p, cudaStreamSynchronize(p->s_in));
    RKL_CK(p, cudaStreamSynchronize(p->stream));
    return rkl_plan_check(p);
}

}  // extern "C"
