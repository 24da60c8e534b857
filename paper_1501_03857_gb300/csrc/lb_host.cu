// C-ABI implementation (include/lb.h): parameter validation, FP64 host
// thermodynamics (critical point, Maxwell coexistence, the EOS pressure),
// the initial pool, workspace layout, launches (plain steps replayed from
// captured graphs), read-back, pressure probes, batches of independent
// instances, and the adjoint driver (checkpoints, segment recomputation
// overlapped with the reverse sweep).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lb.h"
#include "lb_internal.h"

using namespace lbgpu;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(LB_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LB_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------------------------
// Peng-Robinson thermodynamics in FP64 (Eq. 21)
// ---------------------------------------------------------------------------

struct Pr {
    double a, b, R, omega, Tc, kappa;
    explicit Pr(const lb_eos& e)
        : a(e.a), b(e.b), R(e.R), omega(e.omega),
          Tc(0.0778 * e.a / (0.45724 * e.b * e.R)),
          kappa(0.37464 + 1.54226 * e.omega - 0.26992 * e.omega * e.omega) {}
    double phi(double T) const {
        const double t = 1.0 + kappa * (1.0 - std::sqrt(T / Tc));
        return t * t;
    }
    double p(double rho, double T) const {
        return rho * R * T / (1.0 - b * rho) - a * phi(T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
    }
    // integral of p dv in v = 1/rho (antiderivative)
    double prim(double v, double T) const {
        const double s2 = std::sqrt(2.0);
        return R * T * std::log(v - b) -
               a * phi(T) / (2.0 * s2 * b) * std::log((v + b - s2 * b) / (v + b + s2 * b));
    }
};

// root of p(rho) = P on [lo, hi] where p - P changes sign, by bisection
double pr_root(const Pr& e, double T, double P, double lo, double hi) {
    double flo = e.p(lo, T) - P;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        const double fm = e.p(mid, T) - P;
        if ((fm < 0) == (flo < 0)) {
            lo = mid;
            flo = fm;
        } else {
            hi = mid;
        }
        if (hi - lo <= 1e-16 * hi) break;
    }
    return 0.5 * (lo + hi);
}

// Maxwell equal-area construction: find P_sat with p(rho_V) = p(rho_L) =
// P_sat and int_{v_L}^{v_V} (p - P_sat) dv = 0.
int maxwell(const Pr& e, double T, double* rv, double* rl) {
    if (!(T > 0.0 && T < e.Tc)) return fail(LB_E_INVAL, "coexistence needs 0 < T < Tc (T=%g, Tc=%g)", T, e.Tc);
    const int N = 40000;
    const double rmax = (1.0 / e.b) * (1.0 - 1e-9);
    const double r0 = 1e-6, dr = (rmax * 0.999 - r0) / N;
    double r_hi = -1, r_lo = -1, p_hi = 0, p_lo = 0;
    double pprev = e.p(r0, T), dprev = 0;
    for (int i = 1; i <= N; ++i) {
        const double r = r0 + i * dr, pc = e.p(r, T), d = pc - pprev;
        if (i > 1) {
            if (r_hi < 0 && dprev > 0 && d <= 0) { r_hi = r - dr; p_hi = pprev; }
            else if (r_hi > 0 && r_lo < 0 && dprev < 0 && d >= 0) { r_lo = r - dr; p_lo = pprev; break; }
        }
        dprev = d;
        pprev = pc;
    }
    if (r_hi < 0 || r_lo < 0) return fail(LB_E_INVAL, "isotherm T=%g has no van der Waals loop", T);
    p_lo = std::max(p_lo, 1e-8 * p_hi);
    double Plo = p_lo, Phi = p_hi, vV = 0, vL = 0;
    for (int it = 0; it < 300; ++it) {
        const double P = 0.5 * (Plo + Phi);
        const double rV = pr_root(e, T, P, 1e-18, r_hi);
        const double rL = pr_root(e, T, P, r_lo, rmax);
        vV = 1.0 / rV;
        vL = 1.0 / rL;
        const double A = e.prim(vV, T) - e.prim(vL, T) - P * (vV - vL);
        if (A > 0) Plo = P; else Phi = P;
        if (Phi - Plo <= 1e-17 * Phi) break;
    }
    const double P = 0.5 * (Plo + Phi);
    *rv = pr_root(e, T, P, 1e-18, r_hi);
    *rl = pr_root(e, T, P, r_lo, rmax);
    return LB_OK;
}

// ---------------------------------------------------------------------------
// Initial pool (Sec. 3.1) with splitmix64 noise
// ---------------------------------------------------------------------------

inline uint64_t splitmix64(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void pool(int Lx, int Ly, double rl, double rv, double h, double amp, uint64_t seed, float* out) {
    for (int y = 0; y < Ly; ++y) {
        const double prof = 0.5 * (rl + rv) - 0.5 * (rl - rv) * std::tanh(2.0 * (y - h) / 5.0);
        for (int x = 0; x < Lx; ++x) {
            double r = prof;
            if (amp != 0.0) {
                const uint64_t n = (uint64_t)y * (uint64_t)Lx + (uint64_t)x;
                const double u = (double)(splitmix64(seed, n) >> 11) * 0x1.0p-53;
                r = r * (1.0 + amp * (2.0 * u - 1.0));
            }
            out[(size_t)y * Lx + x] = (float)r;
        }
    }
}

int validate(const lb_grid* g, const lb_eos* e, const lb_thermal* t) {
    if (!g || !e || !t) return fail(LB_E_INVAL, "null parameter struct");
    if (g->Lx < 1 || g->Ly < 3) return fail(LB_E_INVAL, "grid %dx%d: need Lx >= 1, Ly >= 3", g->Lx, g->Ly);
    if (g->bc_y < LB_BC_WALLS || g->bc_y > LB_BC_PERIODIC) return fail(LB_E_INVAL, "bad bc_y %d", g->bc_y);
    const long long pitch = (g->Lx + 31) / 32 * 32;
    if (9LL * pitch * g->Ly >= (1LL << 31)) return fail(LB_E_INVAL, "grid too large for 32-bit plane offsets");
    if (!(e->a > 0 && e->b > 0 && e->R > 0)) return fail(LB_E_INVAL, "EOS needs a, b, R > 0");
    if (!(e->G < 0)) return fail(LB_E_INVAL, "G must be negative");
    if (!(e->sigma >= 0)) return fail(LB_E_INVAL, "sigma must be >= 0");
    if (!(t->Ts_over_Tc > 0 && t->Ts_over_Tc < 1)) return fail(LB_E_INVAL, "Ts/Tc must be in (0, 1)");
    if (!(t->cv > 0 && t->cv_chi >= 0)) return fail(LB_E_INVAL, "need cv > 0, cv_chi >= 0");
    if (!(t->nu_l > 0 && t->nu_v > 0)) return fail(LB_E_INVAL, "viscosities must be > 0");
    const double rates[3] = {t->s_e, t->s_zeta, t->s_q};
    for (double r : rates)
        if (!(r > 0 && r < 2)) return fail(LB_E_INVAL, "relaxation rates must be in (0, 2)");
    return LB_OK;
}

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    int pitch;
    size_t plane, f0, f1, t0, t1, thb, acc, qpart, total;
};

// FP64 slots of the per-strip heat-flux sums (the most strips any launch
// shape gives this width)
inline size_t qpart_bytes(int Lx) { return sizeof(double) * (size_t)((Lx + MIN_STRIP_COLS - 1) / MIN_STRIP_COLS); }

Layout layout(const lb_grid* g) {
    Layout L;
    L.pitch = (g->Lx + 31) / 32 * 32;
    L.plane = (size_t)L.pitch * g->Ly;
    const size_t fb = 9 * L.plane * sizeof(float), tb = L.plane * sizeof(float);
    L.f0 = 0;
    L.f1 = align256(L.f0 + fb);
    L.t0 = align256(L.f1 + fb);
    L.t1 = align256(L.t0 + tb);
    L.thb = align256(L.t1 + tb);
    L.acc = align256(L.thb + (size_t)L.pitch * sizeof(float));
    L.qpart = align256(L.acc + sizeof(Acc));
    L.total = align256(L.qpart + qpart_bytes(g->Lx));
    return L;
}

}  // namespace

void lbgpu::set_last_error(const char* msg) { g_err = msg; }

struct lb_handle {
    lb_grid grid;
    lb_eos eos;
    lb_thermal th;
    double Tc, Ts, rho_v, rho_l, rho_ave, Gw, superheat;
    std::vector<double> profile;
    Layout lay;
    char* ws;
    float* f[2];
    float* t[2];
    float* thb;
    Acc* acc;
    double* qpart;
    int cur;
    cudaStream_t st;
    int64_t steps;
    Launch launch;
    StepParams base;
    float* wall_pinned;      // pinned staging of theta_b(x) for the upload
    cudaEvent_t wall_done;   // the last upload from wall_pinned has run
    bool wall_pending;
    // adjoint: private stream for captured segment graphs, keyed by
    // (segment length, lambda parity, scratch base)
    cudaStream_t adj_stream;
    cudaEvent_t adj_in, adj_out;
    cudaStream_t adj_stream2;           // recompute stream of the adjoint
    cudaEvent_t adj_ready[2], adj_free[2];  // segment buffer filled / released
    struct AdjGraph {
        int kind;  // 0: recompute into a segment buffer, 1: reverse sweep over it
        int len, cur, buf, C, nsteps;
        void* scratch;
        StepParams params;  // baked into the graph's kernel nodes
        Launch launch;
        cudaGraphExec_t exec;
    };
    std::vector<AdjGraph> adj_graphs;
    // plain stepping: STEP_GRAPH-step graphs keyed by the parameters of their
    // first step (buffers, accumulators, constants) and the launch shape
    struct StepGraph {
        StepParams first;
        Launch launch;
        ProbeArgs probe;
        cudaGraphExec_t exec;
    };
    std::vector<StepGraph> step_graphs;
    // pressure probes (n = 0: off); f and th are filled per launch
    ProbeArgs probe;
};

namespace {

void fill_params(lb_handle* h) {
    StepParams& P = h->base;
    memset(&P, 0, sizeof(P));
    const lb_grid& g = h->grid;
    const lb_eos& e = h->eos;
    const lb_thermal& t = h->th;
    P.thb = h->thb;
    P.acc = h->acc;
    P.qpart = h->qpart;
    P.Lx = g.Lx;
    P.Ly = g.Ly;
    P.pitch = h->lay.pitch;
    P.plane = (int)h->lay.plane;
    P.bc = g.bc_y;
    P.ghost = g.ghost_layer ? 1 : 0;
    P.isothermal = g.isothermal ? 1 : 0;
    const double kappa = 0.37464 + 1.54226 * e.omega - 0.26992 * e.omega * e.omega;
    P.Ts = (float)h->Ts;
    P.a = (float)e.a;
    P.b = (float)e.b;
    P.R = (float)e.R;
    P.G = (float)e.G;
    P.two_over_G = (float)(2.0 / e.G);
    P.k0 = (float)(1.0 + kappa);
    P.k1 = (float)(kappa / std::sqrt(h->Tc));
    P.k0k1 = (float)((1.0 + kappa) * kappa / std::sqrt(h->Tc));
    P.k1k1 = (float)(kappa * kappa / h->Tc);
    P.s_e = (float)t.s_e;
    P.s_z = (float)t.s_zeta;
    P.s_q = (float)t.s_q;
    P.sig_e = (float)(e.sigma / (1.0 / t.s_e - 0.5));
    P.sig_z = (float)(e.sigma / (1.0 / t.s_zeta - 0.5));
    P.rho_v = (float)h->rho_v;
    P.inv_drho = (float)(1.0 / (h->rho_l - h->rho_v));
    const double tau_v = t.nu_v * 3.0 + 0.5, tau_l = t.nu_l * 3.0 + 0.5;
    P.tau_v = (float)tau_v;
    P.dtau = (float)(tau_l - tau_v);
    P.g = (float)t.g;
    P.rho_ave = (float)h->rho_ave;
    P.gw6 = (float)(h->Gw / 6.0);
    P.chi = (float)(t.cv_chi / t.cv);
    P.cvchi = (float)t.cv_chi;
    P.inv_cv = (float)(1.0 / t.cv);
    set_pairs(P);
}

// The launch shape of the fused step for this grid (block_x, seg_rows 0:
// automatic).
int compute_launch(const lb_handle* h, int block_x, int seg_rows, Launch* out) {
    int dev = 0, nsm = 0;
    LB_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    LB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    const int Lx = h->grid.Lx, Ly = h->grid.Ly;
    // 64 threads up to 4096 columns, 128 beyond (measured: 64 is 1-5 %
    // faster on 1024^2-4096^2, 128 2 % faster on 8192^2)
    int bx = block_x, occ = 0;
    if (bx <= 0) bx = Lx <= 4096 ? 64 : 128;
    if (!dual_supported(bx)) return fail(LB_E_INVAL, "the fused step takes block_x 64, 128 or 256, not %d", bx);
    LB_CUDA(dual_occupancy(bx, &occ), "occupancy");
    if (occ < 1) return fail(LB_E_INVAL, "block_x %d does not fit on an SM", bx);
    const int nout = bx - 2 * HALO;
    const int cols = 2 * nout;  // output columns per block
    const int nstrips = (Lx + cols - 1) / cols;
    int seg = seg_rows;
    if (seg <= 0) {
        const int slots = nsm * occ;
        const int nseg = std::max(1, slots / nstrips);
        seg = std::max(8, (Ly + nseg - 1) / nseg);
    }
    out->block_x = bx;
    out->seg_rows = seg;
    out->nstrips = nstrips;
    out->nseg = (Ly + seg - 1) / seg;
    return LB_OK;
}

// The step parameters that describe launch shape L.
void apply_launch(StepParams& P, const Launch& L) {
    P.nout = L.block_x - 2 * HALO;
    P.nstrips = L.nstrips;
    P.seg_h = L.seg_rows;
}

int choose_launch(lb_handle* h, int block_x, int seg_rows) {
    Launch L;
    const int rc = compute_launch(h, block_x, seg_rows, &L);
    if (rc) return rc;
    h->launch = L;
    apply_launch(h->base, L);
    return LB_OK;
}

// Clear the device fault flags err (read after the stream drained) and map
// them to an error code.
int report_device_errors(lb_handle* h, unsigned err) {
    if (!err) return LB_OK;
    const unsigned z = 0;
    LB_CUDA(cudaMemcpy(&h->acc->err, &z, sizeof(unsigned), cudaMemcpyHostToDevice), "clear error flags");
    if (err & ERR_BOUNDS) return fail(LB_E_BOUNDS, "a device index left its buffer (checked build)");
    if (err & ERR_TIMEOUT)
        return fail(LB_E_TIMEOUT, "a wait of the persistent batch step gave up (its wait limit); the instances' "
                                  "states are only partly advanced");
    if (err & ERR_NONFINITE) return fail(LB_E_NONFINITE, "non-finite density or temperature on the device");
    if (err & ERR_EOS) return fail(LB_E_EOS_DOMAIN, "pseudopotential argument 2(p - rho/3)/G < 0 (EOS domain)");
    return LB_OK;
}

int check_device_errors(lb_handle* h) {
    unsigned err = 0;
    LB_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    LB_CUDA(cudaMemcpy(&err, &h->acc->err, sizeof(unsigned), cudaMemcpyDeviceToHost), "read error flags");
    return report_device_errors(h, err);
}

int upload_wall(lb_handle* h) {
    const int Lx = h->grid.Lx;
    if (h->wall_pending) LB_CUDA(cudaEventSynchronize(h->wall_done), "wait for the previous wall upload");
    for (int x = 0; x < Lx; ++x)
        h->wall_pinned[x] = (float)(h->superheat + (h->profile.empty() ? 0.0 : h->profile[x]));
    LB_CUDA(cudaMemcpyAsync(h->thb, h->wall_pinned, Lx * sizeof(float), cudaMemcpyHostToDevice, h->st),
            "upload wall temperature");
    LB_CUDA(cudaEventRecord(h->wall_done, h->st), "cudaEventRecord");
    h->wall_pending = true;
    return LB_OK;
}

void release(lb_handle* h) {
    if (!h) return;
    if (h->adj_stream) cudaStreamSynchronize(h->adj_stream);
    if (h->adj_stream2) cudaStreamSynchronize(h->adj_stream2);
    for (auto& g : h->adj_graphs) cudaGraphExecDestroy(g.exec);
    for (int k = 0; k < 2; ++k) {
        if (h->adj_ready[k]) cudaEventDestroy(h->adj_ready[k]);
        if (h->adj_free[k]) cudaEventDestroy(h->adj_free[k]);
    }
    if (h->adj_stream2) cudaStreamDestroy(h->adj_stream2);
    for (auto& g : h->step_graphs) cudaGraphExecDestroy(g.exec);
    if (h->adj_in) cudaEventDestroy(h->adj_in);
    if (h->adj_out) cudaEventDestroy(h->adj_out);
    if (h->adj_stream) cudaStreamDestroy(h->adj_stream);
    if (h->wall_pending) cudaEventSynchronize(h->wall_done);
    if (h->wall_done) cudaEventDestroy(h->wall_done);
    if (h->wall_pinned) cudaFreeHost(h->wall_pinned);
    delete h;
}


// ---------------------------------------------------------------------------
// Stepping: runs of STEP_GRAPH steps are replayed from a captured CUDA graph
// on the handle's private stream (ordered after and before the caller's
// stream), the rest are single launches. `P` carries the accumulators and
// constants; its buffers follow h->cur.
// ---------------------------------------------------------------------------

constexpr int STEP_GRAPH = 32;  // even: the buffer parity returns

int aux_stream(lb_handle* h) {
    if (!h->adj_stream) {
        LB_CUDA(cudaStreamCreateWithFlags(&h->adj_stream, cudaStreamNonBlocking), "private stream");
        LB_CUDA(cudaEventCreateWithFlags(&h->adj_in, cudaEventDisableTiming), "private stream event");
        LB_CUDA(cudaEventCreateWithFlags(&h->adj_out, cudaEventDisableTiming), "private stream event");
    }
    return LB_OK;
}

int launch_one(lb_handle* h, const StepParams& base, int cur, cudaStream_t q) {
    StepParams P = base;
    P.f_in = h->f[cur];
    P.f_out = h->f[1 - cur];
    P.th_in = h->t[cur];
    P.th_out = h->t[1 - cur];
    LB_CUDA(launch_step(P, h->launch, q), "step launch");
    if (h->probe.n > 0) {
        ProbeArgs A = h->probe;
        A.f = P.f_out;
        A.th = P.th_in;
        LB_CUDA(launch_probe(A, q), "probe launch");
    }
    return LB_OK;
}

int run_steps(lb_handle* h, const StepParams& base, int nsteps) {
    int left = nsteps;
    if (left >= STEP_GRAPH) {
        int rc = aux_stream(h);
        if (rc) return rc;
        StepParams first = base;
        first.f_in = h->f[h->cur];
        first.f_out = h->f[1 - h->cur];
        first.th_in = h->t[h->cur];
        first.th_out = h->t[1 - h->cur];
        cudaGraphExec_t exec = nullptr;
        for (auto& g : h->step_graphs)
            if (memcmp(&g.first, &first, sizeof(StepParams)) == 0 && memcmp(&g.launch, &h->launch, sizeof(Launch)) == 0 &&
                memcmp(&g.probe, &h->probe, sizeof(ProbeArgs)) == 0)
                exec = g.exec;
        cudaStream_t gs = h->adj_stream;
        if (!exec) {
            cudaGraph_t graph = nullptr;
            LB_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal), "begin capture");
            for (int k = 0; k < STEP_GRAPH && rc == LB_OK; ++k) rc = launch_one(h, base, h->cur ^ (k & 1), gs);
            cudaError_t e = cudaStreamEndCapture(gs, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "step graph");
            if (h->step_graphs.size() >= 8) {
                cudaStreamSynchronize(gs);
                cudaGraphExecDestroy(h->step_graphs.front().exec);
                h->step_graphs.erase(h->step_graphs.begin());
            }
            h->step_graphs.push_back({first, h->launch, h->probe, exec});
        }
        LB_CUDA(cudaEventRecord(h->adj_in, h->st), "cudaEventRecord");
        LB_CUDA(cudaStreamWaitEvent(gs, h->adj_in, 0), "cudaStreamWaitEvent");
        for (; left >= STEP_GRAPH; left -= STEP_GRAPH) {
            LB_CUDA(cudaGraphLaunch(exec, gs), "cudaGraphLaunch");
            h->steps += STEP_GRAPH;
        }
        LB_CUDA(cudaEventRecord(h->adj_out, gs), "cudaEventRecord");
        LB_CUDA(cudaStreamWaitEvent(h->st, h->adj_out, 0), "cudaStreamWaitEvent");
    }
    for (; left > 0; --left) {
        int rc = launch_one(h, base, h->cur, h->st);
        if (rc) return rc;
        h->cur ^= 1;
        h->steps++;
    }
    return LB_OK;
}

}  // namespace

extern "C" {

const char* lb_last_error(void) { return g_err.c_str(); }

int lb_critical_temperature(const lb_eos* eos, double* Tc) {
    if (!eos || !Tc) return fail(LB_E_INVAL, "null argument");
    if (!(eos->a > 0 && eos->b > 0 && eos->R > 0)) return fail(LB_E_INVAL, "EOS needs a, b, R > 0");
    *Tc = Pr(*eos).Tc;
    return LB_OK;
}

int lb_coexistence(const lb_eos* eos, double T, double* rho_v, double* rho_l) {
    if (!eos || !rho_v || !rho_l) return fail(LB_E_INVAL, "null argument");
    if (!(eos->a > 0 && eos->b > 0 && eos->R > 0)) return fail(LB_E_INVAL, "EOS needs a, b, R > 0");
    return maxwell(Pr(*eos), T, rho_v, rho_l);
}

int lb_initial_density(const lb_grid* grid, const lb_eos* eos, const lb_thermal* th, float* rho0) {
    int rc = validate(grid, eos, th);
    if (rc) return rc;
    if (!rho0) return fail(LB_E_INVAL, "null output");
    Pr pr(*eos);
    double rv, rl;
    rc = maxwell(pr, th->Ts_over_Tc * pr.Tc, &rv, &rl);
    if (rc) return rc;
    pool(grid->Lx, grid->Ly, rl, rv, th->pool_height, th->noise_amp, th->seed, rho0);
    return LB_OK;
}

int lb_workspace_bytes(const lb_grid* grid, size_t* bytes) {
    if (!grid || !bytes) return fail(LB_E_INVAL, "null argument");
    if (grid->Lx < 1 || grid->Ly < 3) return fail(LB_E_INVAL, "grid %dx%d: need Lx >= 1, Ly >= 3", grid->Lx, grid->Ly);
    const long long pitch = (grid->Lx + 31) / 32 * 32;
    if (9LL * pitch * grid->Ly >= (1LL << 31)) return fail(LB_E_INVAL, "grid too large for 32-bit plane offsets");
    *bytes = layout(grid).total;
    return LB_OK;
}

int lb_init(lb_handle** out, const lb_grid* grid, const lb_eos* eos, const lb_thermal* th,
            const double* Tb_profile, double superheat, double Gw, const float* rho0, void* dev_workspace,
            size_t workspace_bytes, void* stream) {
    if (!out) return fail(LB_E_INVAL, "null handle pointer");
    *out = nullptr;
    int rc = validate(grid, eos, th);
    if (rc) return rc;
    const Layout lay = layout(grid);
    if (!dev_workspace || workspace_bytes < lay.total)
        return fail(LB_E_INVAL, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, lay.total);
    if (((uintptr_t)dev_workspace) & 255) return fail(LB_E_INVAL, "workspace must be 256-byte aligned");
    if (!std::isfinite(superheat) || !std::isfinite(Gw)) return fail(LB_E_INVAL, "non-finite superheat or Gw");

    lb_handle* h = new lb_handle();
    h->grid = *grid;
    h->eos = *eos;
    h->th = *th;
    Pr pr(*eos);
    h->Tc = pr.Tc;
    h->Ts = th->Ts_over_Tc * pr.Tc;
    rc = maxwell(pr, h->Ts, &h->rho_v, &h->rho_l);
    if (rc) { release(h); return rc; }
    h->Gw = Gw;
    h->superheat = superheat;
    if (Tb_profile) h->profile.assign(Tb_profile, Tb_profile + grid->Lx);
    h->lay = lay;
    h->ws = (char*)dev_workspace;
    h->f[0] = (float*)(h->ws + lay.f0);
    h->f[1] = (float*)(h->ws + lay.f1);
    h->t[0] = (float*)(h->ws + lay.t0);
    h->t[1] = (float*)(h->ws + lay.t1);
    h->thb = (float*)(h->ws + lay.thb);
    h->acc = (Acc*)(h->ws + lay.acc);
    h->qpart = (double*)(h->ws + lay.qpart);
    h->cur = 0;
    h->st = (cudaStream_t)stream;
    h->steps = 0;
    h->wall_pinned = nullptr;
    h->wall_done = nullptr;
    h->wall_pending = false;
    h->adj_stream = nullptr;
    h->adj_in = h->adj_out = nullptr;
    h->adj_stream2 = nullptr;
    h->adj_ready[0] = h->adj_ready[1] = h->adj_free[0] = h->adj_free[1] = nullptr;
    {
        cudaError_t e0 = cudaMallocHost((void**)&h->wall_pinned, grid->Lx * sizeof(float));
        if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&h->wall_done, cudaEventDisableTiming);
        if (e0 != cudaSuccess) {
            release(h);
            return cuda_fail(e0, "wall staging");
        }
    }

    const int Lx = grid->Lx, Ly = grid->Ly;
    std::vector<float> r0;
    const float* src = rho0;
    if (!src) {
        r0.resize((size_t)Lx * Ly);
        pool(Lx, Ly, h->rho_l, h->rho_v, th->pool_height, th->noise_amp, th->seed, r0.data());
        src = r0.data();
    }
    double sum = 0.0;
    for (size_t i = 0; i < (size_t)Lx * Ly; ++i) {
        if (!std::isfinite(src[i]) || src[i] <= 0.f) {
            release(h);
            return fail(LB_E_INVAL, "initial density must be finite and > 0 (cell %zu)", i);
        }
        sum += src[i];
    }
    h->rho_ave = sum / ((double)Lx * Ly);
    fill_params(h);
    cudaError_t e = dual_prepare();
    if (e != cudaSuccess) { release(h); return cuda_fail(e, "cudaFuncSetAttribute"); }
    rc = choose_launch(h, 0, 0);
    if (rc) { release(h); return rc; }

    auto bail = [&](cudaError_t err, const char* what) { release(h); return cuda_fail(err, what); };
    if ((e = cudaMemsetAsync(h->acc, 0, sizeof(Acc), h->st)) != cudaSuccess) return bail(e, "clear accumulators");
    if ((rc = upload_wall(h))) { release(h); return rc; }
    // rho0 goes through the second population buffer as a pitched scratch
    if ((e = cudaMemcpy2DAsync(h->f[1], lay.pitch * sizeof(float), src, Lx * sizeof(float), Lx * sizeof(float), Ly,
                               cudaMemcpyHostToDevice, h->st)) != cudaSuccess)
        return bail(e, "upload rho0");
    StepParams P = h->base;
    if ((e = launch_init(P, h->f[1], h->f[0], h->t[0], h->st)) != cudaSuccess) return bail(e, "init kernel");
    if ((e = cudaStreamSynchronize(h->st)) != cudaSuccess) return bail(e, "lb_init synchronize");
    *out = h;
    return LB_OK;
}

int lb_step(lb_handle* h, int nsteps) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (nsteps < 0) return fail(LB_E_INVAL, "nsteps must be >= 0");
    StepParams P = h->base;
    return run_steps(h, P, nsteps);
}

int lb_set_wall_temperature(lb_handle* h, const double* Tb_profile, double superheat) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (!std::isfinite(superheat)) return fail(LB_E_INVAL, "non-finite superheat");
    h->superheat = superheat;
    if (Tb_profile) h->profile.assign(Tb_profile, Tb_profile + h->grid.Lx);
    else h->profile.clear();
    int rc = upload_wall(h);
    if (rc) return rc;
    if (h->grid.bc_y != LB_BC_PERIODIC)
        LB_CUDA(cudaMemcpyAsync(h->t[h->cur], h->thb, h->grid.Lx * sizeof(float), cudaMemcpyDeviceToDevice, h->st),
                "wall row update");
    return LB_OK;
}

int lb_set_wettability(lb_handle* h, double Gw) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (!std::isfinite(Gw)) return fail(LB_E_INVAL, "non-finite Gw");
    h->Gw = Gw;
    h->base.gw6 = (float)(Gw / 6.0);
    set_pairs(h->base);
    return LB_OK;
}

int lb_heat_flux(lb_handle* h, double* q_inst, double* q_mean, double* q_std, int64_t* nsamples, int reset) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    Acc a;
    // one read of the accumulator record, fault flags included
    LB_CUDA(cudaMemcpyAsync(&a, h->acc, sizeof(Acc), cudaMemcpyDeviceToHost, h->st), "read accumulators");
    LB_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    int rc = report_device_errors(h, a.err);
    const double n = a.q_n;
    const double mean = n > 0 ? a.q_sum / n : 0.0;
    const double var = n > 1 ? std::max(0.0, (a.q_sum2 - n * mean * mean) / (n - 1)) : 0.0;
    if (q_inst) *q_inst = a.q_last;
    if (q_mean) *q_mean = mean;
    if (q_std) *q_std = std::sqrt(var);
    if (nsamples) *nsamples = (int64_t)n;
    if (reset) {
        LB_CUDA(cudaMemsetAsync(&h->acc->q_sum, 0, 3 * sizeof(double), h->st), "reset accumulators");
        LB_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    }
    return rc;
}

int lb_fields(lb_handle* h, float* rho, float* ux, float* uy, float* T, int on_device) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    StepParams P = h->base;
    P.f_in = h->f[h->cur];
    P.th_in = h->t[h->cur];
    float* scr = h->f[1 - h->cur];
    const int Lx = h->grid.Lx, Ly = h->grid.Ly, pitch = h->lay.pitch;
    const size_t pl = h->lay.plane;
    if (on_device) {
        LB_CUDA(launch_macro(P, scr, rho, ux, uy, T, Lx, h->st), "fields kernel");
        return check_device_errors(h);
    }
    float* o[4] = {rho ? scr + 4 * pl : nullptr, ux ? scr + 5 * pl : nullptr, uy ? scr + 6 * pl : nullptr,
                   T ? scr + 7 * pl : nullptr};
    LB_CUDA(launch_macro(P, scr, o[0], o[1], o[2], o[3], pitch, h->st), "fields kernel");
    float* dst[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            LB_CUDA(cudaMemcpy2DAsync(dst[k], Lx * sizeof(float), o[k], pitch * sizeof(float), Lx * sizeof(float), Ly,
                                      cudaMemcpyDeviceToHost, h->st),
                    "fields read-back");
    return check_device_errors(h);
}

int lb_get_state(lb_handle* h, float* fpost, float* theta, int on_device) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    const int Lx = h->grid.Lx, Ly = h->grid.Ly, pitch = h->lay.pitch;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (fpost)
        LB_CUDA(cudaMemcpy2DAsync(fpost, Lx * sizeof(float), h->f[h->cur], pitch * sizeof(float), Lx * sizeof(float),
                                  9 * Ly, k, h->st),
                "populations read-back");
    if (theta)
        LB_CUDA(cudaMemcpy2DAsync(theta, Lx * sizeof(float), h->t[h->cur], pitch * sizeof(float), Lx * sizeof(float),
                                  Ly, k, h->st),
                "temperature read-back");
    return check_device_errors(h);
}

int lb_set_state(lb_handle* h, const float* fpost, const float* theta, int on_device) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    const int Lx = h->grid.Lx, Ly = h->grid.Ly, pitch = h->lay.pitch;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (fpost)
        LB_CUDA(cudaMemcpy2DAsync(h->f[h->cur], pitch * sizeof(float), fpost, Lx * sizeof(float), Lx * sizeof(float),
                                  9 * Ly, k, h->st),
                "populations upload");
    if (theta)
        LB_CUDA(cudaMemcpy2DAsync(h->t[h->cur], pitch * sizeof(float), theta, Lx * sizeof(float), Lx * sizeof(float),
                                  Ly, k, h->st),
                "temperature upload");
    if (!on_device) LB_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_mass(lb_handle* h, double* mass) {
    if (!h || !mass) return fail(LB_E_INVAL, "null argument");
    StepParams P = h->base;
    LB_CUDA(launch_mass(P, h->f[h->cur], h->st), "mass kernel");
    LB_CUDA(cudaMemcpyAsync(mass, &h->acc->mass, sizeof(double), cudaMemcpyDeviceToHost, h->st), "mass read-back");
    return check_device_errors(h);
}

int lb_sync(lb_handle* h) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    return check_device_errors(h);
}

int lb_info(lb_handle* h, int64_t* steps, int* block_x, int* seg_rows, int* nblocks) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (steps) *steps = h->steps;
    if (block_x) *block_x = h->launch.block_x;
    if (seg_rows) *seg_rows = h->launch.seg_rows;
    if (nblocks) *nblocks = h->launch.nstrips * h->launch.nseg;
    return LB_OK;
}

int lb_set_launch(lb_handle* h, int block_x, int seg_rows) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (seg_rows < 0) return fail(LB_E_INVAL, "seg_rows must be >= 0");
    return choose_launch(h, block_x, seg_rows);
}

namespace {
struct SaveHeader {
    char magic[8];
    int32_t Lx, Ly;
    int64_t steps;
    double superheat, Gw;
    int32_t has_profile, pad;
};
}  // namespace

int lb_save_bytes(lb_handle* h, size_t* bytes) {
    if (!h || !bytes) return fail(LB_E_INVAL, "null argument");
    const size_t cells = (size_t)h->grid.Lx * h->grid.Ly;
    *bytes = sizeof(SaveHeader) + sizeof(Acc) + 10 * cells * sizeof(float) + h->grid.Lx * sizeof(double);
    return LB_OK;
}

int lb_save(lb_handle* h, void* host_buf, size_t bytes) {
    size_t need = 0;
    int rc = lb_save_bytes(h, &need);
    if (rc) return rc;
    if (!host_buf || bytes < need) return fail(LB_E_INVAL, "save buffer of %zu bytes < %zu", bytes, need);
    char* p = (char*)host_buf;
    SaveHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "LBBOIL1", 8);
    hd.Lx = h->grid.Lx;
    hd.Ly = h->grid.Ly;
    hd.steps = h->steps;
    hd.superheat = h->superheat;
    hd.Gw = h->Gw;
    hd.has_profile = h->profile.empty() ? 0 : 1;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    LB_CUDA(cudaMemcpyAsync(p, h->acc, sizeof(Acc), cudaMemcpyDeviceToHost, h->st), "save accumulators");
    p += sizeof(Acc);
    const size_t cells = (size_t)h->grid.Lx * h->grid.Ly;
    rc = lb_get_state(h, (float*)p, (float*)p + 9 * cells, 0);
    if (rc) return rc;
    p += 10 * cells * sizeof(float);
    for (int x = 0; x < h->grid.Lx; ++x) ((double*)p)[x] = h->profile.empty() ? 0.0 : h->profile[x];
    return LB_OK;
}

int lb_load(lb_handle* h, const void* host_buf, size_t bytes) {
    size_t need = 0;
    int rc = lb_save_bytes(h, &need);
    if (rc) return rc;
    if (!host_buf || bytes < need) return fail(LB_E_INVAL, "load buffer of %zu bytes < %zu", bytes, need);
    const char* p = (const char*)host_buf;
    SaveHeader hd;
    memcpy(&hd, p, sizeof(hd));
    if (memcmp(hd.magic, "LBBOIL1", 8) != 0 || hd.Lx != h->grid.Lx || hd.Ly != h->grid.Ly)
        return fail(LB_E_INVAL, "checkpoint does not match this grid");
    p += sizeof(hd);
    Acc a;
    memcpy(&a, p, sizeof(Acc));
    a.err = 0;
    a.count = 0;
    LB_CUDA(cudaMemcpyAsync(h->acc, &a, sizeof(Acc), cudaMemcpyHostToDevice, h->st), "load accumulators");
    p += sizeof(Acc);
    const size_t cells = (size_t)h->grid.Lx * h->grid.Ly;
    rc = lb_set_state(h, (const float*)p, (const float*)p + 9 * cells, 0);
    if (rc) return rc;
    p += 10 * cells * sizeof(float);
    h->steps = hd.steps;
    h->Gw = hd.Gw;
    h->base.gw6 = (float)(hd.Gw / 6.0);
    set_pairs(h->base);
    h->superheat = hd.superheat;
    if (hd.has_profile) h->profile.assign((const double*)p, (const double*)p + h->grid.Lx);
    else h->profile.clear();
    rc = upload_wall(h);
    if (rc) return rc;
    LB_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    return LB_OK;
}

int lb_probe_ring_bytes(int n, int capacity, size_t* bytes) {
    if (!bytes) return fail(LB_E_INVAL, "null output");
    if (n < 1 || n > kProbeMax) return fail(LB_E_INVAL, "probe count %d outside 1..%d", n, kProbeMax);
    if (capacity < 1 || capacity > (1 << 26)) return fail(LB_E_INVAL, "probe capacity %d outside 1..2^26", capacity);
    *bytes = 256 + sizeof(float) * 4 * (size_t)n * (size_t)capacity;
    return LB_OK;
}

int lb_set_probes(lb_handle* h, int n, const int* x, const int* y, void* dev_ring, size_t ring_bytes,
                  int capacity) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (n == 0) {
        memset(&h->probe, 0, sizeof(ProbeArgs));
        return LB_OK;
    }
    size_t need = 0;
    int rc = lb_probe_ring_bytes(n, capacity, &need);
    if (rc) return rc;
    if (!x || !y || !dev_ring) return fail(LB_E_INVAL, "null argument");
    if (((uintptr_t)dev_ring) & 255) return fail(LB_E_INVAL, "probe ring must be 256-byte aligned");
    if (ring_bytes < need) return fail(LB_E_INVAL, "probe ring of %zu bytes is smaller than the %zu needed", ring_bytes, need);
    for (int k = 0; k < n; ++k)
        if (x[k] < 0 || x[k] >= h->grid.Lx || y[k] < 0 || y[k] >= h->grid.Ly)
            return fail(LB_E_INVAL, "probe %d at (%d, %d) is outside the %d x %d grid", k, x[k], y[k], h->grid.Lx,
                        h->grid.Ly);
    ProbeArgs A;
    memset(&A, 0, sizeof(A));
    A.ring = (float*)dev_ring;
    A.plane = (int)h->lay.plane;
    A.pitch = h->lay.pitch;
    A.n = n;
    A.cap = capacity;
    for (int k = 0; k < n; ++k) {
        A.x[k] = x[k];
        A.y[k] = y[k];
    }
    const Pr e(h->eos);
    A.a = e.a;
    A.b = e.b;
    A.R = e.R;
    A.Ts = h->Ts;
    A.k0 = 1.0 + e.kappa;
    A.k1 = e.kappa / std::sqrt(e.Tc);
    LB_CUDA(cudaMemsetAsync(dev_ring, 0, 256, h->st), "clear probe ring");
    h->probe = A;
    return LB_OK;
}

int lb_probe_read(lb_handle* h, int max_records, float* out, int64_t* count, int* m_out) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (h->probe.n == 0) return fail(LB_E_INVAL, "no probes are set");
    if (max_records < 0 || (max_records > 0 && !out)) return fail(LB_E_INVAL, "bad output buffer");
    const ProbeArgs& A = h->probe;
    unsigned long long n = 0;
    LB_CUDA(cudaMemcpyAsync(&n, A.ring, sizeof(n), cudaMemcpyDeviceToHost, h->st), "read probe count");
    LB_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
    const long long m = std::min<long long>(std::min<long long>((long long)n, A.cap), max_records);
    if (count) *count = (int64_t)n;
    if (m_out) *m_out = (int)m;
    if (m == 0) return LB_OK;
    std::vector<float> ring((size_t)A.n * A.cap * 4);
    LB_CUDA(cudaMemcpy(ring.data(), A.ring + 64, ring.size() * sizeof(float), cudaMemcpyDeviceToHost),
            "read probe ring");
    for (int k = 0; k < A.n; ++k)
        for (long long j = 0; j < m; ++j) {
            const unsigned long long step = n - (unsigned long long)m + (unsigned long long)j;
            const float* r = &ring[((size_t)k * A.cap + (size_t)(step % (unsigned long long)A.cap)) * 4];
            float* o = out + ((size_t)k * m + (size_t)j) * 3;
            o[0] = r[0];
            o[1] = r[1];
            o[2] = r[2];
        }
    return LB_OK;
}

int lb_eos_pressure(const lb_eos* eos, int64_t n, const float* rho, const float* T, double* p) {
    if (!eos || n < 0 || (n > 0 && (!rho || !T || !p))) return fail(LB_E_INVAL, "null argument");
    if (!(eos->a > 0 && eos->b > 0 && eos->R > 0)) return fail(LB_E_INVAL, "EOS needs a, b, R > 0");
    const Pr e(*eos);
    for (int64_t i = 0; i < n; ++i) p[i] = e.p((double)rho[i], (double)T[i]);
    return LB_OK;
}

int lb_destroy(lb_handle* h) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    release(h);
    return LB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: many independent simulations advanced by one launch per step
// ---------------------------------------------------------------------------

struct lb_batch {
    std::vector<lb_handle*> inst;
    std::vector<size_t> ws_off;  // workspace offset of each instance
    StepParams* table;           // device [2][n]: parameters by step parity
    int* block_off;              // device [n + 1]: first block of each instance
    std::vector<int> h_off;
    std::vector<StepParams> h_table;
    int block_x, seg_req;        // launch shape (seg_req 0: automatic)
    int nblocks;
    bool dirty;                  // tables no longer match the instances' buffers
    int64_t steps;
    cudaStream_t st;             // the caller's stream
    cudaStream_t gs;             // private stream the captured graphs run on
    cudaEvent_t ev_in, ev_out;
    cudaGraphExec_t graph;       // GRAPH_STEPS steps starting at parity 0
    bool kshared;                // all instances share the model constants
    StepParams kconst;           // ... which are these (instance 0's parameters)
    // persistent mode (tpb > 0): one cooperative launch per run of steps, a
    // grid of at most one wave, about tpb tiles per block
    int tpb;
    unsigned long long wait_limit;
    int max_tiles;               // capacity of the tile arrays
    int2* d_tiles;               // device [max_tiles]: (instance, block index)
    int* d_tile_off;             // device [max_tiles + 1]: first tile of each block
    int* d_ntiles;               // device [n]
    unsigned* d_arrive;          // device [n]
    std::vector<int2> h_tiles;
    std::vector<int> h_tile_off, h_ntiles;
    int pgrid;                   // blocks of the persistent launch
    cudaGraphExec_t pgraph;      // PERSIST_STEPS steps in one launch
};

namespace {

constexpr int GRAPH_STEPS = 32;  // steps per captured graph (even: parity returns)
constexpr int PERSIST_STEPS = 32;  // steps per persistent launch in the captured graph (even)
constexpr unsigned long long PERSIST_WAIT_DEFAULT = 1ull << 24;  // polls (64 ns sleeps): about 1-2 s

size_t batch_tail_offset(const lb_batch_desc* d, int n, std::vector<size_t>* offs) {
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        if (offs) offs->push_back(off);
        off += layout(&d[i].grid).total;
    }
    return off;
}

// Most tiles a batch can have: the 64-thread blocks' strips (the narrowest)
// and segments of one row.
long long batch_max_tiles(const lb_batch_desc* d, int n) {
    long long t = 0;
    for (int i = 0; i < n; ++i)
        t += (long long)((d[i].grid.Lx + MIN_STRIP_COLS - 1) / MIN_STRIP_COLS) * d[i].grid.Ly;
    return t;
}

// Byte offsets of the batch's device arrays after the instances' workspaces.
struct BatchTail {
    size_t table, block_off, tiles, tile_off, ntiles, arrive, total;
};

BatchTail batch_tail(const lb_batch_desc* d, int n) {
    BatchTail T;
    const long long mt = batch_max_tiles(d, n);
    T.table = align256(batch_tail_offset(d, n, nullptr));
    T.block_off = align256(T.table + 2 * n * sizeof(StepParams));
    T.tiles = align256(T.block_off + (n + 1) * sizeof(int));
    T.tile_off = align256(T.tiles + (size_t)mt * sizeof(int2));
    T.ntiles = align256(T.tile_off + (size_t)(mt + 1) * sizeof(int));
    T.arrive = align256(T.ntiles + n * sizeof(int));
    T.total = align256(T.arrive + n * sizeof(unsigned));
    return T;
}

// The model constants the step reads from K (step_body, lb_step3.cu): the
// float2 pairs except the wettability and rho_ave, inv_drho, rho_v, cvchi.
bool same_constants(const StepParams& a, const StepParams& b) {
    for (int k = 0; k < KP_COUNT; ++k)
        if (k != KP_GW6 && k != KP_RHOAVE && memcmp(&a.kp[k], &b.kp[k], sizeof(float2)) != 0) return false;
    return a.inv_drho == b.inv_drho && a.rho_v == b.rho_v && a.cvchi == b.cvchi;
}

// Whether every instance shares instance 0's model constants; if so the step
// takes them from its parameters (lb_step_batch_k) instead of each block's
// shared-memory copy.
void batch_constants(lb_batch* b) {
    b->kconst = b->inst[0]->base;
    b->kshared = true;
    for (lb_handle* h : b->inst)
        if (!same_constants(h->base, b->kconst)) b->kshared = false;
}

// Common block size, per-instance segment height and block offsets. With an
// automatic segment height every instance gets a share of one full wave
// proportional to its cells (tpb waves' worth in the persistent mode, whose
// grid is one wave that takes about tpb tiles per block).
int batch_layout(lb_batch* b) {
    const int n = (int)b->inst.size();
    int dev = 0, nsm = 0, occ = 0;
    LB_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    LB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    batch_constants(b);
    if (b->tpb > 0) LB_CUDA(persist_occupancy(b->block_x, b->kshared, &occ), "occupancy");
    else LB_CUDA(batch_occupancy(b->block_x, b->kshared, &occ), "occupancy");
    if (occ < 1) return fail(LB_E_INVAL, "batch block_x %d does not fit on an SM", b->block_x);
    const int waves = std::max(1, b->tpb);
    const int nout = b->block_x - 2 * HALO;
    // Without a requested height every tile gets about the same number of
    // rows: a block costs its rows (plus the pipeline's halo) whatever share
    // of its columns the instance fills, and the step lasts as long as its
    // longest tile. S is the smallest height at which the tiles still fit in
    // `waves` waves; an instance splits its rows into ceil(Ly / S) equal
    // segments.
    auto nstrips_of = [&](const lb_handle* h) { return (h->grid.Lx + 2 * nout - 1) / (2 * nout); };
    int S = 8;
    if (b->seg_req <= 0) {
        const long long cap = (long long)nsm * occ * waves;
        auto tiles_at = [&](int height) {
            long long t = 0;
            for (lb_handle* h : b->inst) t += (long long)nstrips_of(h) * ((h->grid.Ly + height - 1) / height);
            return t;
        };
        int hi = 8;
        for (lb_handle* h : b->inst) hi = std::max(hi, h->grid.Ly);
        while (S < hi) {  // the smallest height whose tiles fit (tiles_at falls as the height grows)
            const int mid = S + (hi - S) / 2;
            if (tiles_at(mid) <= cap) hi = mid;
            else S = mid + 1;
        }
    }
    b->h_off.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        lb_handle* h = b->inst[i];
        const int nstrips = nstrips_of(h);
        int seg = b->seg_req;
        if (seg <= 0) {
            const int nseg = (h->grid.Ly + S - 1) / S;
            seg = (h->grid.Ly + nseg - 1) / nseg;
        }
        h->launch.block_x = b->block_x;
        h->launch.seg_rows = seg;
        h->launch.nstrips = nstrips;
        h->launch.nseg = (h->grid.Ly + seg - 1) / seg;
        h->base.nout = nout;
        h->base.nstrips = nstrips;
        h->base.seg_h = seg;
        b->h_off[i + 1] = b->h_off[i] + nstrips * h->launch.nseg;
    }
    b->nblocks = b->h_off[n];
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->pgraph) {
        cudaGraphExecDestroy(b->pgraph);
        b->pgraph = nullptr;
    }
    LB_CUDA(cudaMemcpyAsync(b->block_off, b->h_off.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->st),
            "batch offsets upload");
    if (b->tpb > 0) {
        // Deal the tiles out to a grid of at most one wave, longest first to
        // the least loaded block (a tile costs its rows plus the pipeline's
        // 10 rows of halo); each block then takes its tiles in (instance,
        // tile) order, the same order on every block.
        const int ntile = b->nblocks;
        if (ntile > b->max_tiles) return fail(LB_E_INVAL, "batch has %d tiles, more than the %d provided for", ntile, b->max_tiles);
        const int G = std::min(ntile, nsm * occ);
        std::vector<std::pair<int, int>> order;  // (cost, tile)
        std::vector<int2> tiles(ntile);
        b->h_ntiles.assign(n, 0);
        for (int i = 0; i < n; ++i) {
            lb_handle* h = b->inst[i];
            const int nt = b->h_off[i + 1] - b->h_off[i];
            b->h_ntiles[i] = nt;
            for (int k = 0; k < nt; ++k) {
                const int seg = k / h->launch.nstrips;
                const int rows = std::min(h->launch.seg_rows, h->grid.Ly - seg * h->launch.seg_rows);
                tiles[b->h_off[i] + k] = make_int2(i, k);
                order.push_back({rows + 2 * HALO, b->h_off[i] + k});
            }
        }
        std::stable_sort(order.begin(), order.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) {
            return x.first > y.first;
        });
        std::vector<long long> load(G, 0);
        std::vector<std::vector<int>> mine(G);
        std::vector<std::pair<long long, int>> heap;  // (load, block), a min-heap
        for (int g = 0; g < G; ++g) heap.push_back({0, g});
        auto cmp = [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) { return x > y; };
        for (const auto& o : order) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto& top = heap.back();
            top.first += o.first;
            mine[top.second].push_back(o.second);
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
        // blocks in the order of their first tile (for one tile per block,
        // the order of the per-step launch), so that the costly tiles LPT
        // dealt out first do not sit on consecutive blocks
        for (auto& m : mine) std::sort(m.begin(), m.end());  // tile ids are ordered by (instance, tile)
        std::sort(mine.begin(), mine.end(), [](const std::vector<int>& x, const std::vector<int>& y) {
            return x.front() < y.front();
        });
        b->h_tiles.clear();
        b->h_tile_off.assign(1, 0);
        for (int g = 0; g < G; ++g) {
            for (int t : mine[g]) b->h_tiles.push_back(tiles[t]);
            b->h_tile_off.push_back((int)b->h_tiles.size());
        }
        b->pgrid = G;
        LB_CUDA(cudaMemcpyAsync(b->d_tiles, b->h_tiles.data(), ntile * sizeof(int2), cudaMemcpyHostToDevice, b->st),
                "tiles upload");
        LB_CUDA(cudaMemcpyAsync(b->d_tile_off, b->h_tile_off.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice,
                                b->st),
                "tile offsets upload");
        LB_CUDA(cudaMemcpyAsync(b->d_ntiles, b->h_ntiles.data(), n * sizeof(int), cudaMemcpyHostToDevice, b->st),
                "tile counts upload");
    }
    b->dirty = true;
    return LB_OK;
}

// Parameter tables relative to each instance's current buffer: parity p
// reads buffer cur ^ p. Uploaded in stream order (cudaMemcpyAsync from
// pageable host memory stages the source before it returns).
int batch_upload(lb_batch* b) {
    if (!b->dirty) return LB_OK;
    const int n = (int)b->inst.size();
    b->h_table.resize(2 * n);
    for (int p = 0; p < 2; ++p)
        for (int i = 0; i < n; ++i) {
            lb_handle* h = b->inst[i];
            StepParams P = h->base;
            const int c = h->cur ^ p;
            P.f_in = h->f[c];
            P.f_out = h->f[1 - c];
            P.th_in = h->t[c];
            P.th_out = h->t[1 - c];
            b->h_table[p * n + i] = P;
        }
    LB_CUDA(cudaMemcpyAsync(b->table, b->h_table.data(), 2 * n * sizeof(StepParams), cudaMemcpyHostToDevice, b->st),
            "batch table upload");
    b->dirty = false;
    return LB_OK;
}

int batch_launch_one(lb_batch* b, cudaStream_t s, int parity) {
    const int n = (int)b->inst.size();
    LB_CUDA(batch_launch(b->block_x, b->table + parity * n, b->block_off, n, b->nblocks,
                         b->kshared ? &b->kconst : nullptr, s),
            "batch step launch");
    return LB_OK;
}

// One persistent launch of `nsteps` steps (the arrival counters zeroed first).
int persist_launch_one(lb_batch* b, cudaStream_t s, int nsteps) {
    const int n = (int)b->inst.size();
    PersistArgs A;
    A.table = b->table;
    A.tiles = b->d_tiles;
    A.tile_off = b->d_tile_off;
    A.ntiles = b->d_ntiles;
    A.arrive = b->d_arrive;
    A.n = n;
    A.nsteps = nsteps;
    A.wait_limit = b->wait_limit;
    LB_CUDA(cudaMemsetAsync(b->d_arrive, 0, n * sizeof(unsigned), s), "clear arrival counters");
    LB_CUDA(persist_launch(b->block_x, b->kshared ? &b->kconst : nullptr, A, b->pgrid, s), "persistent batch launch");
    return LB_OK;
}

int persist_graph(lb_batch* b, cudaGraphExec_t* out) {
    if (!b->pgraph) {
        cudaGraph_t g = nullptr;
        LB_CUDA(cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal), "begin capture");
        int rc = persist_launch_one(b, b->gs, PERSIST_STEPS);
        cudaError_t e = cudaStreamEndCapture(b->gs, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&b->pgraph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    }
    *out = b->pgraph;
    return LB_OK;
}

int batch_graph(lb_batch* b, cudaGraphExec_t* out) {
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        LB_CUDA(cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal), "begin capture");
        int rc = LB_OK;
        for (int k = 0; k < GRAPH_STEPS && rc == LB_OK; ++k) rc = batch_launch_one(b, b->gs, k & 1);
        cudaError_t e = cudaStreamEndCapture(b->gs, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    }
    *out = b->graph;
    return LB_OK;
}

void batch_release(lb_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->gs) cudaStreamSynchronize(b->gs);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->gs) cudaStreamDestroy(b->gs);
    for (lb_handle* h : b->inst) release(h);
    delete b;
}

}  // namespace

extern "C" {

int lb_batch_workspace_bytes(const lb_batch_desc* d, int n, size_t* bytes) {
    if (!d || n < 1 || !bytes) return fail(LB_E_INVAL, "need n >= 1 descriptors and an output");
    for (int i = 0; i < n; ++i)
        if (d[i].grid.Lx < 1 || d[i].grid.Ly < 3) return fail(LB_E_INVAL, "instance %d: grid too small", i);
    *bytes = batch_tail(d, n).total;
    return LB_OK;
}

int lb_batch_init(lb_batch** out, const lb_batch_desc* d, int n, void* dev_workspace, size_t workspace_bytes,
                  void* stream) {
    if (!out) return fail(LB_E_INVAL, "null batch pointer");
    *out = nullptr;
    size_t need = 0;
    int rc = lb_batch_workspace_bytes(d, n, &need);
    if (rc) return rc;
    if (!dev_workspace || workspace_bytes < need)
        return fail(LB_E_INVAL, "batch workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, need);
    if (((uintptr_t)dev_workspace) & 255) return fail(LB_E_INVAL, "workspace must be 256-byte aligned");
    lb_batch* b = new lb_batch();
    b->table = nullptr;
    b->block_off = nullptr;
    b->graph = nullptr;
    b->st = (cudaStream_t)stream;
    b->gs = nullptr;
    b->ev_in = b->ev_out = nullptr;
    b->steps = 0;
    b->block_x = 128;
    b->seg_req = 0;
    b->dirty = true;
    b->tpb = 0;
    b->wait_limit = PERSIST_WAIT_DEFAULT;
    b->pgrid = 0;
    b->pgraph = nullptr;
    b->d_tiles = nullptr;
    b->d_tile_off = b->d_ntiles = nullptr;
    b->d_arrive = nullptr;
    char* ws = (char*)dev_workspace;
    const size_t tail = batch_tail_offset(d, n, &b->ws_off);
    for (int i = 0; i < n; ++i) {
        lb_handle* h = nullptr;
        rc = lb_init(&h, &d[i].grid, &d[i].eos, &d[i].th, d[i].Tb_profile, d[i].superheat, d[i].Gw, d[i].rho0,
                     ws + b->ws_off[i], layout(&d[i].grid).total, stream);
        if (rc) {
            const std::string msg = g_err;
            batch_release(b);
            return fail(rc, "instance %d: %s", i, msg.c_str());
        }
        b->inst.push_back(h);
    }
    const BatchTail T = batch_tail(d, n);
    (void)tail;
    b->table = (StepParams*)(ws + T.table);
    b->block_off = (int*)(ws + T.block_off);
    b->d_tiles = (int2*)(ws + T.tiles);
    b->d_tile_off = (int*)(ws + T.tile_off);
    b->d_ntiles = (int*)(ws + T.ntiles);
    b->d_arrive = (unsigned*)(ws + T.arrive);
    b->max_tiles = (int)std::min<long long>(batch_max_tiles(d, n), INT32_MAX);
    cudaError_t e = batch_prepare();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        batch_release(b);
        return cuda_fail(e, "batch set-up");
    }
    rc = batch_layout(b);
    if (rc == LB_OK) rc = batch_upload(b);
    if (rc == LB_OK && (e = cudaStreamSynchronize(b->st)) != cudaSuccess) rc = cuda_fail(e, "batch init sync");
    if (rc) {
        batch_release(b);
        return rc;
    }
    *out = b;
    return LB_OK;
}

int lb_batch_set_launch(lb_batch* b, int block_x, int seg_rows) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    if (!batch_supported(block_x)) return fail(LB_E_INVAL, "batch block_x must be 64 or 128, not %d", block_x);
    if (seg_rows < 0) return fail(LB_E_INVAL, "seg_rows must be >= 0");
    b->block_x = block_x;
    b->seg_req = seg_rows;
    return batch_layout(b);
}

int lb_batch_set_persistent(lb_batch* b, int tiles_per_block, long long wait_limit) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    if (tiles_per_block < 0 || tiles_per_block > 64) return fail(LB_E_INVAL, "tiles_per_block must be in 0..64");
    b->tpb = tiles_per_block;
    b->wait_limit = wait_limit > 0 ? (unsigned long long)wait_limit : PERSIST_WAIT_DEFAULT;
    return batch_layout(b);
}

int lb_batch_step(lb_batch* b, int nsteps) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    if (nsteps < 0) return fail(LB_E_INVAL, "nsteps must be >= 0");
    int rc = batch_upload(b);
    if (rc) return rc;
    int left = nsteps, parity = 0;
    if (b->tpb > 0) {
        // runs of PERSIST_STEPS steps: one persistent launch each, replayed
        // from a captured graph on the private stream; the rest in one launch
        if (left >= PERSIST_STEPS) {
            cudaGraphExec_t g = nullptr;
            rc = persist_graph(b, &g);
            if (rc) return rc;
            LB_CUDA(cudaEventRecord(b->ev_in, b->st), "cudaEventRecord");
            LB_CUDA(cudaStreamWaitEvent(b->gs, b->ev_in, 0), "cudaStreamWaitEvent");
            for (; left >= PERSIST_STEPS; left -= PERSIST_STEPS) LB_CUDA(cudaGraphLaunch(g, b->gs), "cudaGraphLaunch");
            LB_CUDA(cudaEventRecord(b->ev_out, b->gs), "cudaEventRecord");
            LB_CUDA(cudaStreamWaitEvent(b->st, b->ev_out, 0), "cudaStreamWaitEvent");
        }
        if (left > 0 && (rc = persist_launch_one(b, b->st, left))) return rc;
        left = 0;
    }
    if (left >= GRAPH_STEPS) {
        // whole chunks as a captured graph on the private stream, ordered
        // after and before the caller's stream
        cudaGraphExec_t g = nullptr;
        rc = batch_graph(b, &g);
        if (rc) return rc;
        LB_CUDA(cudaEventRecord(b->ev_in, b->st), "cudaEventRecord");
        LB_CUDA(cudaStreamWaitEvent(b->gs, b->ev_in, 0), "cudaStreamWaitEvent");
        for (; left >= GRAPH_STEPS; left -= GRAPH_STEPS) LB_CUDA(cudaGraphLaunch(g, b->gs), "cudaGraphLaunch");
        LB_CUDA(cudaEventRecord(b->ev_out, b->gs), "cudaEventRecord");
        LB_CUDA(cudaStreamWaitEvent(b->st, b->ev_out, 0), "cudaStreamWaitEvent");
    }
    for (; left > 0; --left, parity ^= 1) {
        rc = batch_launch_one(b, b->st, parity);
        if (rc) return rc;
    }
    for (lb_handle* h : b->inst) {
        h->cur ^= (nsteps & 1);
        h->steps += nsteps;
    }
    if (nsteps & 1) b->dirty = true;  // tables follow each instance's current buffer
    b->steps += nsteps;
    return LB_OK;
}

// Every instance is read (and its fault flags cleared); the first failure
// is returned.
int lb_batch_heat_flux(lb_batch* b, double* q_inst, double* q_mean, double* q_std, int64_t* nsamples, int reset) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    int first = LB_OK;
    std::string msg;
    for (size_t i = 0; i < b->inst.size(); ++i) {
        int rc = lb_heat_flux(b->inst[i], q_inst ? q_inst + i : nullptr, q_mean ? q_mean + i : nullptr,
                              q_std ? q_std + i : nullptr, nsamples ? nsamples + i : nullptr, reset);
        if (rc && first == LB_OK) {
            first = rc;
            msg = g_err;
        }
    }
    if (first) g_err = msg;
    return first;
}

int lb_batch_get_state(lb_batch* b, int i, float* fpost, float* theta, int on_device) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return fail(LB_E_INVAL, "bad batch or instance index");
    return lb_get_state(b->inst[i], fpost, theta, on_device);
}

int lb_batch_fields(lb_batch* b, int i, float* rho, float* ux, float* uy, float* T, int on_device) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return fail(LB_E_INVAL, "bad batch or instance index");
    return lb_fields(b->inst[i], rho, ux, uy, T, on_device);
}

int lb_batch_set_state(lb_batch* b, int i, const float* fpost, const float* theta, int on_device) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return fail(LB_E_INVAL, "bad batch or instance index");
    return lb_set_state(b->inst[i], fpost, theta, on_device);
}

int lb_batch_set_wall_temperature(lb_batch* b, int i, const double* Tb_profile, double superheat) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return fail(LB_E_INVAL, "bad batch or instance index");
    return lb_set_wall_temperature(b->inst[i], Tb_profile, superheat);
}

int lb_batch_set_wettability(lb_batch* b, int i, double Gw) {
    if (!b || i < 0 || i >= (int)b->inst.size()) return fail(LB_E_INVAL, "bad batch or instance index");
    int rc = lb_set_wettability(b->inst[i], Gw);
    if (rc == LB_OK) b->dirty = true;
    return rc;
}

int lb_batch_info(lb_batch* b, int64_t* steps, int* block_x, int* nblocks) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    if (steps) *steps = b->steps;
    if (block_x) *block_x = b->block_x;
    if (nblocks) *nblocks = b->tpb > 0 ? b->pgrid : b->nblocks;
    return LB_OK;
}

int lb_batch_sync(lb_batch* b) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    int first = LB_OK;
    std::string msg;
    for (lb_handle* h : b->inst) {
        int rc = check_device_errors(h);
        if (rc && first == LB_OK) {
            first = rc;
            msg = g_err;
        }
    }
    if (first) g_err = msg;
    return first;
}

int lb_batch_destroy(lb_batch* b) {
    if (!b) return fail(LB_E_INVAL, "null batch");
    batch_release(b);
    return LB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradients of the window-averaged wall heat flux (discrete adjoint)
// ---------------------------------------------------------------------------

namespace {

struct AdjLayout {
    size_t work, acc, lam, ckpt, seg, rec, total;
    int nck;
};

AdjLayout adj_layout(const lb_handle* h, const StepParams& P, int nsteps, int C) {
    AdjLayout L;
    const size_t state = align256(sizeof(float) * 10 * (size_t)P.plane);
    L.nck = nsteps / C + 1;
    L.work = 0;
    L.acc = align256(L.work + adjoint_work_bytes(P));
    L.lam = align256(L.acc + sizeof(Acc));
    L.ckpt = L.lam + 2 * align256(sizeof(float) * 11 * (size_t)P.plane);  // lambda: lf, theta, lr
    L.seg = L.ckpt + (size_t)L.nck * state;
    L.rec = L.seg + 2 * (size_t)C * state;  // two segment buffers of states
    // and of the forward intermediates of each of their steps; with a
    // checkpoint every step, the intermediates of every step instead
    const size_t nrec = C == 1 ? (size_t)nsteps : 2 * (size_t)C;
    L.total = L.rec + nrec * align256(sizeof(float) * kRecomputePlanes * (size_t)P.plane);
    (void)h;
    return L;
}

int adjoint_check(lb_handle* h, int nsteps, int C) {
    if (!h) return fail(LB_E_INVAL, "null handle");
    if (nsteps < 1 || C < 1) return fail(LB_E_INVAL, "need nsteps >= 1 and ckpt_every >= 1");
    if (h->grid.bc_y == LB_BC_PERIODIC || h->grid.isothermal)
        return fail(LB_E_INVAL, "the adjoint supports wall-bounded or outflow-top thermal runs only");
    return LB_OK;
}

}  // namespace

extern "C" {

int lb_adjoint_scratch_bytes(lb_handle* h, int nsteps, int ckpt_every, size_t* bytes) {
    int rc = adjoint_check(h, nsteps, ckpt_every);
    if (rc) return rc;
    if (!bytes) return fail(LB_E_INVAL, "null output");
    *bytes = adj_layout(h, h->base, nsteps, ckpt_every).total;
    return LB_OK;
}

int lb_adjoint_pick_ckpt(lb_handle* h, int nsteps, size_t budget_bytes, int* ckpt_every, size_t* bytes) {
    int rc = adjoint_check(h, nsteps, 1);
    if (rc) return rc;
    if (!ckpt_every) return fail(LB_E_INVAL, "null output");
    const size_t all = adj_layout(h, h->base, nsteps, 1).total;
    int pick = 1;
    size_t need = all;
    if (all > budget_bytes) {
        // checkpoints fall as 1/C and the replay buffers grow as C: the
        // smallest scratch lies near C = sqrt(nsteps / 4), well inside C*C <= nsteps + 16
        pick = 0;
        for (long long c = 2; c <= nsteps && c * c <= (long long)nsteps + 16; ++c) {
            const size_t t = adj_layout(h, h->base, nsteps, (int)c).total;
            if (pick == 0 || t < need) {
                pick = (int)c;
                need = t;
            }
        }
        if (pick == 0 || need > budget_bytes)
            return fail(LB_E_INVAL, "no checkpoint interval fits the adjoint of %d steps in %zu bytes (smallest: %zu)",
                        nsteps, budget_bytes, pick ? need : all);
    }
    *ckpt_every = pick;
    if (bytes) *bytes = need;
    return LB_OK;
}

int lb_adjoint(lb_handle* h, int nsteps, int ckpt_every, void* dev_scratch, size_t scratch_bytes, double* J,
               double* dJ_dTb, double* dJ_dGw) {
    int rc = adjoint_check(h, nsteps, ckpt_every);
    if (rc) return rc;
    const int C = ckpt_every;
    const StepParams base = h->base;
    const AdjLayout L = adj_layout(h, base, nsteps, C);
    if (!dev_scratch || scratch_bytes < L.total)
        return fail(LB_E_INVAL, "adjoint scratch of %zu bytes is smaller than the %zu needed", scratch_bytes, L.total);
    if (((uintptr_t)dev_scratch) & 255) return fail(LB_E_INVAL, "scratch must be 256-byte aligned");
    char* s = (char*)dev_scratch;
    const size_t pl = (size_t)base.plane;
    const size_t state = align256(sizeof(float) * 10 * pl);
    void* work = s + L.work;
    Acc* acc = (Acc*)(s + L.acc);
    auto sf = [&](size_t off, int k) { return (float*)(s + off + (size_t)k * state); };
    // adjoint state, twice: lf (9 planes), lambda_theta, lr (lb_internal.h)
    const size_t lam_state = align256(sizeof(float) * 11 * pl);
    float* lam[2] = {(float*)(s + L.lam), (float*)(s + L.lam + lam_state)};
    cudaStream_t st = h->st;

    // forward: nsteps steps from the current state, J = mean q(t), checkpoints
    LB_CUDA(cudaMemsetAsync(acc, 0, sizeof(Acc), st), "clear adjoint accumulators");
    auto save = [&](float* dst, const float* f, const float* t) -> int {
        LB_CUDA(cudaMemcpyAsync(dst, f, sizeof(float) * 9 * pl, cudaMemcpyDeviceToDevice, st), "checkpoint copy");
        LB_CUDA(cudaMemcpyAsync(dst + 9 * pl, t, sizeof(float) * pl, cudaMemcpyDeviceToDevice, st),
                "checkpoint copy");
        return LB_OK;
    };
    if ((rc = save(sf(L.ckpt, 0), h->f[h->cur], h->t[h->cur]))) return rc;
    const size_t rec_stride = align256(sizeof(float) * kRecomputePlanes * pl);
    auto rec_at = [&](size_t k) {  // the k-th set of forward intermediates
        float* r = (float*)(s + L.rec + k * rec_stride);
        return RecomputeOut{r,          r + pl,     r + 2 * pl, r + 3 * pl, r + 4 * pl,
                            r + 5 * pl, r + 6 * pl, r + 7 * pl, r + 8 * pl, r + 9 * pl};
    };
    if (C == 1) {
        // every step stored: the forward pass runs the fused step in its
        // recompute mode with the step's output and q(t), writing state n+1
        // into checkpoint n+1 and the step's intermediates into set n, so the
        // reverse sweep replays nothing
        for (int n = 0; n < nsteps; ++n) {
            StepParams P = base;
            P.acc = acc;
            P.f_in = sf(L.ckpt, n);
            P.th_in = sf(L.ckpt, n) + 9 * pl;
            P.f_out = sf(L.ckpt, n + 1);
            P.th_out = sf(L.ckpt, n + 1) + 9 * pl;
            LB_CUDA(dual_recompute(P, rec_at(n), true, true, h->launch, st), "adjoint forward step");
            if (h->probe.n > 0) {
                ProbeArgs A = h->probe;
                A.f = P.f_out;
                A.th = P.th_in;
                LB_CUDA(launch_probe(A, st), "probe launch");
            }
        }
        // the simulation advances as with the plain steps: the last state
        // into the current population and theta buffers (separate arrays of
        // the workspace, not one 10-plane block like a checkpoint)
        LB_CUDA(cudaMemcpyAsync(h->f[h->cur], sf(L.ckpt, nsteps), sizeof(float) * 9 * pl, cudaMemcpyDeviceToDevice,
                                st),
                "state copy");
        LB_CUDA(cudaMemcpyAsync(h->t[h->cur], sf(L.ckpt, nsteps) + 9 * pl, sizeof(float) * pl,
                                cudaMemcpyDeviceToDevice, st),
                "state copy");
        h->steps += nsteps;
    } else {
        StepParams P = base;
        P.acc = acc;
        for (int n0 = 0; n0 < nsteps; n0 += C) {
            const int len = std::min(C, nsteps - n0);
            if ((rc = run_steps(h, P, len))) return rc;
            if (n0 + len == nsteps) break;
            if ((rc = save(sf(L.ckpt, (n0 + len) / C), h->f[h->cur], h->t[h->cur]))) return rc;
        }
    }
    Acc a;
    LB_CUDA(cudaMemcpyAsync(&a, acc, sizeof(Acc), cudaMemcpyDeviceToHost, st), "read J");
    LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (a.err & ERR_BOUNDS) return fail(LB_E_BOUNDS, "a device index left its buffer in the window (checked build)");
    if (a.err & ERR_NONFINITE) return fail(LB_E_NONFINITE, "non-finite density or temperature in the window");
    if (a.err & ERR_EOS) return fail(LB_E_EOS_DOMAIN, "pseudopotential argument < 0 in the window (EOS domain)");
    const double Jv = a.q_n > 0 ? a.q_sum / a.q_n : 0.0;
    const float lq = (float)(1.0 / nsteps);

    // reverse: segments from the last checkpoint back to the first. Segment
    // k is recomputed from its checkpoint into one of two buffers on one
    // private stream while the reverse sweep of segment k + 1 runs on another;
    // both are captured CUDA graphs.
    LB_CUDA(cudaMemsetAsync(lam[0], 0, lam_state, st), "clear lambda");
    LB_CUDA(adjoint_grads_reset(base, work, st), "clear gradients");
    if ((rc = aux_stream(h))) return rc;
    if (!h->adj_stream2) {
        LB_CUDA(cudaStreamCreateWithFlags(&h->adj_stream2, cudaStreamNonBlocking), "adjoint stream");
        for (int b2 = 0; b2 < 2; ++b2) {
            LB_CUDA(cudaEventCreateWithFlags(&h->adj_ready[b2], cudaEventDisableTiming), "adjoint event");
            LB_CUDA(cudaEventCreateWithFlags(&h->adj_free[b2], cudaEventDisableTiming), "adjoint event");
        }
    }
    cudaStream_t rs = h->adj_stream;   // reverse sweeps
    cudaStream_t cs = h->adj_stream2;  // recomputation
    LB_CUDA(cudaEventRecord(h->adj_in, st), "cudaEventRecord");
    LB_CUDA(cudaStreamWaitEvent(rs, h->adj_in, 0), "cudaStreamWaitEvent");
    LB_CUDA(cudaStreamWaitEvent(cs, h->adj_in, 0), "cudaStreamWaitEvent");
    auto seg_state = [&](int buf, int j) { return sf(L.seg, buf * C + j); };
    auto seg_rec = [&](int buf, int j) { return rec_at((size_t)(buf * C + j)); };  // step j of buffer buf
    // A segment is replayed from its checkpoint by the fused step in its
    // recompute mode: each step writes the next state and its own forward
    // intermediates (the last writes only the intermediates), so the reverse
    // steps need no recomputation of their own.
    auto recompute = [&](int len, int buf, cudaStream_t q) -> int {
        for (int j = 0; j < len; ++j) {
            StepParams P = base;
            P.acc = acc;
            P.f_in = seg_state(buf, j);
            P.th_in = seg_state(buf, j) + 9 * pl;
            const bool out = j + 1 < len;
            P.f_out = out ? seg_state(buf, j + 1) : nullptr;
            P.th_out = out ? seg_state(buf, j + 1) + 9 * pl : nullptr;
            LB_CUDA(dual_recompute(P, seg_rec(buf, j), out, false, h->launch, q), "adjoint recompute step");
        }
        return LB_OK;
    };
    const StepParams RB = base;
    auto sweep = [&](int len, int buf, int c0, cudaStream_t q) -> int {
        int c = c0;
        for (int j = len - 1; j >= 0; --j) {
            const float* fs = seg_state(buf, j);
            LB_CUDA(adjoint_reverse_step(RB, seg_rec(buf, j), work, fs, fs + 9 * pl, lam[c], lam[c] + 9 * pl,
                                         lam[c] + 10 * pl, lam[1 - c], lam[1 - c] + 9 * pl, lam[1 - c] + 10 * pl, lq, q),
                    "adjoint reverse step");
            c ^= 1;
        }
        return LB_OK;
    };
    // every step stored (C = 1): one sweep over all of them, each reading its
    // state and intermediates where the forward pass left them
    auto sweep_all = [&](cudaStream_t q) -> int {
        int c = 0;
        for (int j = nsteps - 1; j >= 0; --j) {
            const float* fs = sf(L.ckpt, j);
            LB_CUDA(adjoint_reverse_step(RB, rec_at((size_t)j), work, fs, fs + 9 * pl, lam[c], lam[c] + 9 * pl,
                                         lam[c] + 10 * pl, lam[1 - c], lam[1 - c] + 9 * pl, lam[1 - c] + 10 * pl, lq, q),
                    "adjoint reverse step");
            c ^= 1;
        }
        return LB_OK;
    };
    // kind 0: replay of a segment, 1: reverse sweep over a segment, 2: the
    // sweep over every stored step
    auto graph_of = [&](int kind, int len, int buf, int c0, cudaStream_t q, cudaGraphExec_t* out) -> int {
        for (auto& g : h->adj_graphs)
            if (g.kind == kind && g.len == len && g.buf == buf && g.cur == c0 && g.C == C && g.nsteps == nsteps &&
                g.scratch == dev_scratch && memcmp(&g.params, &base, sizeof(StepParams)) == 0 &&
                memcmp(&g.launch, &h->launch, sizeof(Launch)) == 0) {
                *out = g.exec;
                return LB_OK;
            }
        cudaGraph_t graph = nullptr;
        LB_CUDA(cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal), "begin capture");
        int r = kind == 0 ? recompute(len, buf, q) : kind == 1 ? sweep(len, buf, c0, q) : sweep_all(q);
        cudaError_t e = cudaStreamEndCapture(q, &graph);
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint graph");
        if (h->adj_graphs.size() >= 16) {
            cudaStreamSynchronize(rs);
            cudaStreamSynchronize(cs);
            cudaGraphExecDestroy(h->adj_graphs.front().exec);
            h->adj_graphs.erase(h->adj_graphs.begin());
        }
        h->adj_graphs.push_back({kind, len, c0, buf, C, nsteps, dev_scratch, base, h->launch, exec});
        *out = exec;
        return LB_OK;
    };
    const int kmax = (nsteps - 1) / C;
    auto fill = [&](int k) -> int {  // recompute segment k into buffer k & 1
        const int buf = k & 1, len = std::min(C, nsteps - k * C);
        if (k + 2 <= kmax) LB_CUDA(cudaStreamWaitEvent(cs, h->adj_free[buf], 0), "cudaStreamWaitEvent");
        LB_CUDA(cudaMemcpyAsync(seg_state(buf, 0), sf(L.ckpt, k), sizeof(float) * 10 * pl, cudaMemcpyDeviceToDevice,
                                cs),
                "checkpoint copy");
        {
            cudaGraphExec_t g = nullptr;
            int r = graph_of(0, len, buf, 0, cs, &g);
            if (r) return r;
            LB_CUDA(cudaGraphLaunch(g, cs), "cudaGraphLaunch");
        }
        LB_CUDA(cudaEventRecord(h->adj_ready[buf], cs), "cudaEventRecord");
        return LB_OK;
    };
    int cur = 0;
    if (C == 1) {
        cudaGraphExec_t g = nullptr;
        if ((rc = graph_of(2, nsteps, 0, 0, rs, &g))) return rc;
        LB_CUDA(cudaGraphLaunch(g, rs), "cudaGraphLaunch");
        cur = nsteps & 1;
    } else if ((rc = fill(kmax))) {
        return rc;
    }
    for (int k = C == 1 ? -1 : kmax; k >= 0; --k) {
        const int buf = k & 1, len = std::min(C, nsteps - k * C);
        if (k > 0 && (rc = fill(k - 1))) return rc;  // overlaps the sweep below
        LB_CUDA(cudaStreamWaitEvent(rs, h->adj_ready[buf], 0), "cudaStreamWaitEvent");
        cudaGraphExec_t g = nullptr;
        if ((rc = graph_of(1, len, buf, cur, rs, &g))) return rc;
        LB_CUDA(cudaGraphLaunch(g, rs), "cudaGraphLaunch");
        LB_CUDA(cudaEventRecord(h->adj_free[buf], rs), "cudaEventRecord");
        cur ^= (len & 1);
    }
    LB_CUDA(cudaEventRecord(h->adj_out, rs), "cudaEventRecord");
    LB_CUDA(cudaStreamWaitEvent(st, h->adj_out, 0), "cudaStreamWaitEvent");
    LB_CUDA(cudaStreamWaitEvent(cs, h->adj_out, 0), "cudaStreamWaitEvent");
    double dGw = 0.0;
    LB_CUDA(adjoint_grads_finish(base, work, lam[cur] + 9 * pl, dJ_dTb, &dGw, st), "read gradients");
    LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (J) *J = Jv;
    if (dJ_dGw) *dJ_dGw = dGw;
    return check_device_errors(h);
}

}  // extern "C"
