// Discrete adjoint of one time step (reverse mode), for gradients of the
// time-averaged bottom-wall heat flux J = (1/S) sum_n q(t_n) (Sec. 3.2) with
// respect to the wall temperature profile T_b(x) and the wettability G_w of
// Eq. 22.
//
// Forward intermediates of step n are recomputed from the stored state
// (f*^n, theta^n) by the fused step itself in its recompute mode
// (lb_step3.cu, RecomputeOut), which the adjoint driver runs while it
// replays a checkpoint segment. The reverse passes then transpose each part
// of the step in the opposite order:
//
//   RK4 of Eq. 18 (stage 4 .. 1)   -> lambda_theta, lambda of the per-cell
//   and the coefficients              coefficients (ax, ay, cA, cB), then
//   (rev_thermal_fused: one           lambda of grad rho and div v, and the
//   column-marching launch)           local parts of lambda_rho, lambda_v
//   MRT collision (Eqs. 2, 5, 8), v (Eq. 6), forces (Eqs. 7, 9, 22),
//   pull-streaming (Eq. 3)         -> lambda_f*^n without the lambda_rho
//   (rev_flow_fused, stage C)         share, lambda_psi, lambda_F_m
//   F_m neighbour sums (Eq. 7), psi (Eq. 21), q_w, rho = sum f
//   (rev_flow_fused, stage P)      -> lambda_rho (shared by all nine pulled
//                                     populations: carried to the next
//                                     reverse step as one plane), lambda_theta;
//                                     on the wall rows the Zou-He fill and the
//                                     pull transposed with it
//
// A stencil applied forward as out(x) = sum_d c_d in(x + d) is transposed as
// a gather lambda_in(y) += sum_d c_d lambda_out(y - d). Fields are pitched
// [Ly][pitch] FP32; gradients are accumulated in FP64. Supported: walls in
// y or the outflow top, with or without the ghost layer (the host checks).
#include <algorithm>

#include "lb_internal.h"

namespace lbgpu {

namespace {

// Reciprocal, 1/sqrt and sqrt (of a positive value) from single
// special-function instructions (PTX rcp.approx, rsqrt.approx: relative
// error about 1e-7, well inside the adjoint's FP32 budget).
__device__ __forceinline__ float rcp_a(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rsqrt_a(float a) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ constexpr int EXd[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__device__ constexpr int EYd[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Global accesses of the reverse kernels: element i of an array of n. In the
// checked build (LB_CHECKED) an index outside [0, n) sets ERR_BOUNDS in the
// launch's fault flags; a load then reads element 0 instead (an index
// select, not a branch, so the arithmetic around it compiles as in the
// normal build) and a store is skipped. The kernels name their parameter
// struct P.
#ifdef LB_CHECKED
__device__ __forceinline__ bool adj_inside(const StepParams& P, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(&P.acc->err, ERR_BOUNDS);
    return false;
}
#define LB_LD(p, i, n) ((p)[adj_inside(P, (long long)(i), (long long)(n)) ? (long long)(i) : 0LL])
#define LB_ST(p, i, n, v)                                             \
    do {                                                              \
        if (adj_inside(P, (long long)(i), (long long)(n))) (p)[i] = (v); \
    } while (0)
#define LB_ADD(p, i, n, v)                                             \
    do {                                                               \
        if (adj_inside(P, (long long)(i), (long long)(n))) (p)[i] += (v); \
    } while (0)
#else
#define LB_LD(p, i, n) ((p)[i])
#define LB_ST(p, i, n, v) ((p)[i] = (v))
#define LB_ADD(p, i, n, v) ((p)[i] += (v))
#endif

// All the field planes one adjoint step works on.
struct AdjFields {
    // forward intermediates of the step being reversed (RecomputeOut)
    const float* fstar;  // f*^n, 9 planes
    const float* theta;  // theta^n
    const float *rho, *psi;
    const float *drx, *dry, *divv, *ax, *ay;
    const float *u2, *u3, *u4;
    // adjoints; lambda of f* is carried as lf[a](t) + lr(t + e_a) (see
    // adjoint_reverse_step in lb_internal.h)
    const float* lf_in;  // lf part of lambda of f*^{n+1}, 9 planes
    const float* lt_in;  // lambda of theta^{n+1}
    const float* lr_in;  // lr part of lambda of f*^{n+1}
    float* lf_out;       // lf part of lambda of f*^n, 9 planes
    float* lt_out;       // lambda of theta^n
    float* lr_out;       // lr part of lambda of f*^n
    float* sb;           // lambda of the pulled populations of the two wall rows: [9][2][pitch]
    float *lrho, *lvx, *lvy, *lth;  // the thermal pass's parts
    float *ldrx, *ldry, *ldivv;
    double* dTb;   // [Lx] dJ/d theta_b accumulators
    double* dGwx;  // [Lx] dJ/dG_w contributions of each column's first fluid row
    double* dGw;   // dJ/dG_w (sum of dGwx, formed at the end)
};

// p_EOS and its partial derivatives (Eq. 21), FP32.
struct Eos {
    float p, p_rho, p_T, phi, dphi;
};

__device__ __forceinline__ Eos eos(float rho, float T, const StepParams& P) {
    const float rs = rsqrt_a(T), sT = T * rs;
    const float base = P.k0 - P.k1 * sT;  // 1 + kappa (1 - sqrt(T / Tc))
    const float phi = base * base;
    const float dphi = P.k1k1 - P.k0k1 * rs;  // phi'(T)
    const float br = P.b * rho;
    const float i1 = rcp_a(1.f - br);
    const float D = 1.f + 2.f * br - br * br;
    const float iD = rcp_a(D);
    const float dD = 2.f * P.b - 2.f * P.b * br;  // dD/drho
    Eos e;
    e.p = rho * P.R * T * i1 - P.a * phi * rho * rho * iD;
    e.p_rho = P.R * T * i1 * i1 - P.a * phi * rho * (2.f * D - rho * dD) * iD * iD;
    e.p_T = rho * P.R * i1 - P.a * dphi * rho * rho * iD;
    e.phi = phi;
    e.dphi = dphi;
    return e;
}

// ---- reverse -----------------------------------------------------------------

// coefficients -> lambda of grad rho, div v (local) and the local parts of
// lambda_rho, lambda_v, for cell i (after the last stage's accumulation)
// (rho, divv, drx, dry: the cell's forward values)
__device__ __forceinline__ void rev_coef_vals(const StepParams& P, const AdjFields& A, int i, bool wall, float lax,
                                              float lay, float lcA, float lcB, float rho, float divv, float drx,
                                              float dry) {
    if (wall) {
        LB_ST(A.ldrx, i, P.plane, 0.f);
        LB_ST(A.ldry, i, P.plane, 0.f);
        LB_ST(A.ldivv, i, P.plane, 0.f);
        LB_ST(A.lrho, i, P.plane, 0.f);
        LB_ST(A.lvx, i, P.plane, 0.f);
        LB_ST(A.lvy, i, P.plane, 0.f);
        return;
    }
    const float irho = rcp_a(rho);
    const float br = P.b * rho;
    const float i1 = rcp_a(1.f - br);
    const float D = 1.f + 2.f * br - br * br, iD = rcp_a(D);
    const float dD = 2.f * P.b - 2.f * P.b * br;
    LB_ST(A.ldrx, i, P.plane, P.chi * lax * irho);
    LB_ST(A.ldry, i, P.plane, P.chi * lay * irho);
    LB_ST(A.ldivv, i, P.plane, lcA * P.R * P.inv_cv * i1 + lcB * P.a * rho * P.inv_cv * iD);
    LB_ST(A.lrho, i, P.plane,
          -P.chi * (drx * lax + dry * lay) * irho * irho + lcA * divv * P.R * P.inv_cv * P.b * i1 * i1 +
              lcB * divv * P.a * P.inv_cv * (D - rho * dD) * iD * iD);
    LB_ST(A.lvx, i, P.plane, -lax);
    LB_ST(A.lvy, i, P.plane, -lay);
}

// ---- the four RK stages transposed in one column-marching launch ------------
//
// Each RK stage of Eq. 18 (stage 4 .. 1) transposed and then the
// coefficients (rev_coef_vals), cell by cell, in one pass over the domain: a
// block of RT_BD threads owns RT_BD - 2 RT_HALO output columns and a segment
// of rows and marches up the segment one row per iteration, each thread one
// column:
//
//   S  row L    : mu4 = lambda_theta'/6 (fluid rows), ax, ay into shared
//                 rings; u4, u3 (row L), u2 (row L - 2), theta (row L - 3);
//                 cA, cB, lambda-bar (own column)
//   R4 row L-1  : stage 4 transposed (rows L-2..L) -> mu3
//   R3 row L-2  : stage 3 transposed -> mu2
//   R2 row L-3  : stage 2 transposed -> mu1
//   R1 row L-4  : stage 1 transposed; the cell's coefficient adjoints are
//                 complete: lambda of grad rho, div v, rho, v, theta out
//
// A stage's lambda_u at x gathers c_d(x - d) mu(x - d) over the 9 cells
// around x, with c_d(s) = ax(s) wx(d) + ay(s) wy(d) + chi wl(d) the
// isotropic stencils of Sec. 2. With the first-derivative weights odd in d
// that is lambda_u = -Dx[ax mu] - Dy[ay mu] + chi Lap[mu]: the forward
// stencils applied to the products, formed at each neighbour from the ax,
// ay and mu rings (ax, ay are the same for all four stages, so two rings
// serve them all). Each stage reaches one column further out: 4
// halo columns per side. The per-cell accumulators (coefficient adjoints,
// lambda_theta) ride along with their row in registers. Walls in y only
// (the adjoint's supported case). (Measured: this scalar form with 4 warps
// per block runs 1.5 x faster than a paired-FP32 form over two strips,
// whose shared rings allowed only 10 warps per SM; rings of the products
// ax mu, ay mu per stage took 43.5 KB per block, 5 blocks per SM. Steady
// iterations without range and wall tests: 95 registers, 5 blocks per SM,
// and the 2048^2 reverse step 0.374 ms instead of 0.414; held to 7 blocks
// per SM, 72 registers with a small spill, 0.414. Packing each stage's u,
// mu, ax mu and ay mu into one float4 ring, products formed by the thread
// that forms mu, so that a neighbour is one 16-byte load (9 loads and 2
// products per stage instead of 33 and 12): 0.404 ms at 4 blocks per SM
// (128 registers), 0.446 at 5 (96 registers with a spill), against 0.363
// for this form: a 16-byte load of a warp takes 4 shared-memory wavefronts
// and the partial float4 stores at a 16-byte stride as many, more than the
// 33 conflict-free 4-byte loads they replace.)
// ring rows: RT_R for mu and u (3 rows read, one written per iteration),
// RT_RA for ax, ay (read by all four stages: rows L-5..L)
constexpr int RT_BD = 128, RT_HALO = 4, RT_W = RT_BD + 2, RT_R = 4, RT_RA = 8;
constexpr int RT_SMN = (8 * RT_R + 2 * RT_RA) * RT_W + 3 * RT_R * RT_BD;  // floats of shared memory

__global__ void __launch_bounds__(RT_BD) rev_thermal_fused(const StepParams P, AdjFields A, int seg_h) {
    extern __shared__ float rt_sm[];
    float* const sMU = rt_sm;                   // per stage (4, 3, 2, 1 -> 0..3): [4][RT_R][RT_W]
    float* const sU = sMU + 4 * RT_R * RT_W;    // u4, u3, u2, theta: [4][RT_R][RT_W]
    float* const sAX = sU + 4 * RT_R * RT_W;    // ax, ay: [2][RT_RA][RT_W]
    float* const sOWN = sAX + 2 * RT_RA * RT_W;  // cA, cB, lambda-bar: [3][RT_R][RT_BD]
    constexpr int SMN = RT_SMN;
    for (int i = threadIdx.x; i < SMN; i += RT_BD) rt_sm[i] = 0.f;

    const int Lx = P.Lx, Ly = P.Ly, pitch = P.pitch;
    const int nout = RT_BD - 2 * RT_HALO;
    const int nstrips = (Lx + nout - 1) / nout;
    const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
    const int lc = threadIdx.x, s = lc + 1;
    int x = (strip * nout - RT_HALO + lc) % Lx;
    if (x < 0) x += Lx;
    const bool out = lc >= RT_HALO && lc < RT_HALO + nout && strip * nout + lc - RT_HALO < Lx;
    const int ys = seg * seg_h, ye = min(ys + seg_h, Ly);
    const int lo = max(ys - RT_HALO, 0), hi = min(ye + RT_HALO - 1, Ly - 1);  // rows loaded
    const float chi = P.chi;
    // this thread's slot of row L - j in the rings, j = 0..5, set at the
    // start of iteration L; a ring field is a fixed offset from it, so every
    // shared access is a register plus an immediate
    float* p4[6] = {};  // mu and u rings (RT_R slots)
    float* p8[6] = {};  // ax, ay rings (RT_RA slots)
    float* q4[6] = {};  // own-column values (RT_R slots)
    auto own = [&](int f, int j) -> float& { return q4[j][f * RT_R * RT_BD]; };  // 0 cA, 1 cB, 2 lambda-bar
    auto mu = [&](int k, int j) { return p4[j] + k * RT_R * RT_W; };
    auto uu = [&](int k, int j) { return p4[j] + (4 + k) * RT_R * RT_W; };
    auto aring = [&](int k, int j) { return p8[j] + k * RT_RA * RT_W; };  // 0 ax, 1 ay
    float acc_ax[4], acc_ay[4], acc_cA[4], acc_cB[4], acc_th[4];  // index k: the row stage k worked on
#pragma unroll
    for (int k = 0; k < 4; ++k) acc_ax[k] = acc_ay[k] = acc_cA[k] = acc_cB[k] = acc_th[k] = 0.f;
    __syncthreads();

    // stage k (0: stage 4 .. 3: stage 1) at row r = L - 1 - k (slot k + 1;
    // its rows r - 1 and r + 1 are slots k + 2 and k); in a steady iteration
    // (S) no row of any stage is a wall row or next to one
    auto stage = [&](const int k, const int r, auto steady) {
        constexpr bool S = decltype(steady)::value;
        const bool wall = !S && (r == 0 || r == Ly - 1);
        // rows beyond the walls hold no cell: their products are 0
        const bool hm = S || r - 1 >= 0, hp = S || r + 1 < Ly;
        const int jm = k + 2, jc = k + 1, jp = k;
        const float* xm = aring(0, jm);
        const float* xc = aring(0, jc);
        const float* xp = aring(0, jp);
        const float* ym = aring(1, jm);
        const float* yp = aring(1, jp);
        const float* mm = mu(k, jm);
        const float* mc = mu(k, jc);
        const float* mp = mu(k, jp);
        // 12 Dx[ax mu], 12 Dy[ay mu], 6 Lap[mu] (unweighted sums of the stencils)
        float dxp = 4.f * (xc[1] * mc[1] - xc[-1] * mc[-1]), dyp = 0.f;
        float lap = -20.f * mc[0] + 4.f * (mc[1] + mc[-1]);
        if (hm) {
            dxp += xm[1] * mm[1] - xm[-1] * mm[-1];
            dyp -= 4.f * ym[0] * mm[0] + ym[1] * mm[1] + ym[-1] * mm[-1];
            lap += 4.f * mm[0] + mm[1] + mm[-1];
        }
        if (hp) {
            dxp += xp[1] * mp[1] - xp[-1] * mp[-1];
            dyp += 4.f * yp[0] * mp[0] + yp[1] * mp[1] + yp[-1] * mp[-1];
            lap += 4.f * mp[0] + mp[1] + mp[-1];
        }
        float lu = -(dxp + dyp) * (1.f / 12.f) + chi * (1.f / 6.f) * lap;
        const float m = mc[0];
        float lax = 0.f, lay = 0.f, lcA = 0.f, lcB = 0.f;
        if (!wall && m != 0.f) {
            const float* um = uu(k, jm);
            const float* uc = uu(k, jc);
            const float* up = uu(k, jp);
            const float T = P.Ts + uc[0];
            const float rsq = rsqrt_a(T);
            const float dphi = P.k1k1 - P.k0k1 * rsq;
            const float d2phi = 0.5f * P.k0k1 * (rsq * rsq * rsq);
            const float cA = own(0, jc), cB = own(1, jc);
            lu += (-(cA - cB * dphi) + T * cB * d2phi) * m;
            const float ux = (uc[1] - uc[-1]) * (1.f / 3.f) + ((up[1] - um[-1]) + (um[1] - up[-1])) * (1.f / 12.f);
            const float uy = (up[0] - um[0]) * (1.f / 3.f) + ((up[1] - um[-1]) + (up[-1] - um[1])) * (1.f / 12.f);
            lax = ux * m;
            lay = uy * m;
            lcA = -T * m;
            lcB = T * dphi * m;
        }
        if (k == 0) {
            acc_ax[0] = lax;
            acc_ay[0] = lay;
            acc_cA[0] = lcA;
            acc_cB[0] = lcB;
            acc_th[0] = own(2, jc) + lu;
        } else {
            acc_ax[k] += lax;
            acc_ay[k] += lay;
            acc_cA[k] += lcA;
            acc_cB[k] += lcB;
            acc_th[k] += lu;
        }
        if (k < 3) {  // the next stage's mu = a lambda-bar + b lambda_u on fluid rows
            const float ab = k == 2 ? 1.f / 6.f : 1.f / 3.f, bb = k == 0 ? 1.f : 0.5f;
            *mu(k + 1, jc) = wall ? 0.f : ab * own(2, jc) + bb * lu;
        }
    };

    // the inputs of iteration L, loaded one iteration ahead (their latency is
    // hidden behind the stages): lambda_theta', ax, ay, u4, u3 of row L, rho
    // and div v of row L - 1 (for cA, cB), u2 of row L - 2, theta of row
    // L - 3, and rho, div v, grad rho of row L - 4 (the output row)
    float n_lin = 0.f, n_ax = 0.f, n_ay = 0.f, n_u4 = 0.f, n_u3 = 0.f, n_r1 = 0.f, n_d1 = 0.f, n_u2 = 0.f, n_th = 0.f;
    float n_rho = 0.f, n_dv = 0.f, n_drx = 0.f, n_dry = 0.f;
    auto prefetch = [&](int L, auto steady) {
        constexpr bool S = decltype(steady)::value;
        if (S || L <= hi) {
            const int i = L * pitch + x;
            n_lin = LB_LD(A.lt_in, i, P.plane);
            n_ax = LB_LD(A.ax, i, P.plane);
            n_ay = LB_LD(A.ay, i, P.plane);
            n_u4 = LB_LD(A.u4, i, P.plane);
            n_u3 = LB_LD(A.u3, i, P.plane);
        }
        if (S || (L - 1 >= lo && L - 1 <= hi)) {
            const int i = (L - 1) * pitch + x;
            n_r1 = LB_LD(A.rho, i, P.plane);
            n_d1 = LB_LD(A.divv, i, P.plane);
        }
        if (S || (L - 2 >= lo && L - 2 <= hi)) n_u2 = LB_LD(A.u2, (L - 2) * pitch + x, P.plane);
        if (S || (L - 3 >= lo && L - 3 <= hi)) n_th = LB_LD(A.theta, (L - 3) * pitch + x, P.plane);
        if ((S || (L - 4 >= ys && L - 4 < ye)) && out) {
            const int i = (L - 4) * pitch + x;
            n_rho = LB_LD(A.rho, i, P.plane);
            n_dv = LB_LD(A.divv, i, P.plane);
            n_drx = LB_LD(A.drx, i, P.plane);
            n_dry = LB_LD(A.dry, i, P.plane);
        }
    };
    prefetch(lo, std::false_type{});
    // one row iteration L; in a steady one (S) every row it touches (L - 5 ..
    // L + 1) is loaded, off the walls and not next to them, and the output
    // row is the block's own, so the range and wall tests are compiled out
    auto iter = [&](const int L, auto steady) {
        constexpr bool S = decltype(steady)::value;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            p4[j] = rt_sm + ((L - j) & (RT_R - 1)) * RT_W + s;
            p8[j] = sAX + ((L - j) & (RT_RA - 1)) * RT_W + s;
            q4[j] = sOWN + ((L - j) & (RT_R - 1)) * RT_BD + lc;
        }
        // ---- S: the prefetched row into the rings, then the next one's loads
        if (S || L <= hi) {
            const bool wall = !S && (L == 0 || L == Ly - 1);
            *mu(0, 0) = wall ? 0.f : n_lin * (1.f / 6.f);
            *aring(0, 0) = n_ax;
            *aring(1, 0) = n_ay;
            own(2, 0) = wall ? 0.f : n_lin;
            *uu(0, 0) = n_u4;
            *uu(1, 0) = n_u3;
        }
        if (S || (L - 1 >= lo && L - 1 <= hi)) {  // cA, cB of row L - 1 (stage 4 there next)
            // the coefficients of the source term as the step forms them (Eq. 18):
            // cA = div v R / (c_v (1 - b rho)), cB = div v a rho / (c_v (1 + 2 b rho - b^2 rho^2))
            const float br = P.b * n_r1;
            own(0, 1) = n_d1 * P.R * P.inv_cv * rcp_a(1.f - br);
            own(1, 1) = n_d1 * P.a * n_r1 * P.inv_cv * rcp_a(fmaf(br, 2.f - br, 1.f));
        }
        if (S || (L - 2 >= lo && L - 2 <= hi)) *uu(2, 2) = n_u2;
        if (S || (L - 3 >= lo && L - 3 <= hi)) *uu(3, 3) = n_th;
        const float o_rho = n_rho, o_dv = n_dv, o_drx = n_drx, o_dry = n_dry;  // row L - 4
        prefetch(L + 1, steady);
        __syncthreads();
        if (S || (L - 1 >= lo && L - 1 <= hi)) stage(0, L - 1, steady);
        __syncthreads();
        if (S || (L - 2 >= lo && L - 2 <= hi)) stage(1, L - 2, steady);
        __syncthreads();
        if (S || (L - 3 >= lo && L - 3 <= hi)) stage(2, L - 3, steady);
        __syncthreads();
        const int r = L - 4;
        if (S || (r >= ys && r < ye)) {
            stage(3, r, steady);
            if (out) {
                const int i = r * pitch + x;
                LB_ST(A.lth, i, P.plane, acc_th[3]);
                rev_coef_vals(P, A, i, !S && (r == 0 || r == Ly - 1), acc_ax[3], acc_ay[3], acc_cA[3], acc_cB[3],
                              o_rho, o_dv, o_drx, o_dry);
                if (!S && r == 0) LB_ADD(A.dTb, x, P.pitch, (double)LB_LD(A.lt_in, i, P.plane));
            }
        }
#pragma unroll
        for (int k = 3; k > 0; --k) {
            acc_ax[k] = acc_ax[k - 1];
            acc_ay[k] = acc_ay[k - 1];
            acc_cA[k] = acc_cA[k - 1];
            acc_cB[k] = acc_cB[k - 1];
            acc_th[k] = acc_th[k - 1];
        }
        __syncthreads();
    };
    // steady iterations: the rows L - 5 .. L + 1 lie in [1, Ly - 2] and in
    // the loaded rows, the output rows of L and L + 1 in [ys, ye)
    const int Ls = max(max(ys + 4, 6), lo + 1);
    const int Le = min(min(hi - 1, Ly - 2), ye + 2) + 1;
    int L = lo;
    for (; L < Ls; ++L) iter(L, std::false_type{});
    for (; L < Le; ++L) iter(L, std::true_type{});
    for (; L <= hi + RT_HALO; ++L) iter(L, std::false_type{});
}

constexpr size_t rt_smem_bytes() { return sizeof(float) * (size_t)RT_SMN; }

// ---- collision, forces, psi and the pull transposed in one column-marching launch
//
// A block of RF_BD threads owns RF_BD - 2 RF_HALO output columns and a
// segment of rows and marches up it, each thread one column, two stages per
// row iteration L:
//
//   C  row L    : the gathers of the RK-coefficient gradients (lambda_rho +=
//                 -(Dx[ldrx] + Dy[ldry]), lambda_v += -D[ldivv]), the MRT
//                 collision (additive form f* = f + M^-1 dm), velocity and the
//                 local force terms transposed, cell by cell. rho, j and v
//                 are formed again from the pulled populations (as the step
//                 forms them), F from F_m, psi and rho. The cell's lambda of
//                 the pulled populations, without the lambda_rho share, goes
//                 straight through the transposed pull into lf_out (wall
//                 rows: into sb for stage P); psi lambda_F_m goes to a ring.
//   P  row L-1  : F_m's neighbour sums transposed (Eq. 7): with Q = psi
//                 lambda_F_m at the source cell and the first-derivative
//                 weights odd, lambda_psi += G (Dx[Qx] + Dy[Qy]); then psi
//                 (Eq. 21), q(t) (Sec. 3.2) and rho = sum f transposed:
//                 lambda_rho of the cell, shared by all nine pulled
//                 populations, goes to lr_out (read by the next reverse step
//                 where it reads lf); on the wall rows it is added to the
//                 populations in sb, the Zou-He fill is transposed and the
//                 result is pulled back into lf_out. lambda_theta out.
//
// The stencil inputs (ldrx, ldry, ldivv and lr_in of rows L-1..L+1 for C,
// Q of rows L-2..L for P) sit in shared rings; every other input of row L+1
// is loaded into registers during row L. C reaches one column further out
// than its own and P one more: 2 halo columns per side. The owner's own
// share of F_m(x) = -G psi(x) sum_a w_a psi(x + e_a) e_a is (F_m . lambda_F_m)
// / psi; where psi = 0 (outside the EOS domain, which the forward step flags)
// it is taken as 0. Steady iterations are compiled without the range and
// wall tests; held to 4 blocks per SM (128 registers) that measured 1 %
// faster than before the split, 3 blocks per SM (145 registers) 2 % slower.
constexpr int RF_BD = 128, RF_HALO = 2, RF_W = RF_BD + 2, RF_R = 4;

// 12 Dx[v], 12 Dy[v] of a shared ring around lane pointer c (rows m, c, p)
__device__ __forceinline__ void grad12(const float* m, const float* c, const float* p, float& dx, float& dy) {
    dx = 4.f * (c[1] - c[-1]) + (p[1] - p[-1]) + (m[1] - m[-1]);
    dy = 4.f * (p[0] - m[0]) + (p[1] - m[1]) + (p[-1] - m[-1]);
}

__global__ void __launch_bounds__(RF_BD, 4) rev_flow_fused(const StepParams P, AdjFields A, float lq, int seg_h) {
    // rings: 0 ldrx, 1 ldry, 2 ldivv, 3 lr_in, 6 psi (rows of stage C), 4 Qx,
    // 5 Qy (stage P)
    __shared__ float sm[7 * RF_R * RF_W];
    for (int k = threadIdx.x; k < 7 * RF_R * RF_W; k += RF_BD) sm[k] = 0.f;
    const int Lx = P.Lx, Ly = P.Ly, pitch = P.pitch, pl = P.plane;
    const int nout = RF_BD - 2 * RF_HALO;
    const int nstrips = (Lx + nout - 1) / nout;
    const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
    const int lc = threadIdx.x, s = lc + 1;
    int x = (strip * nout - RF_HALO + lc) % Lx;
    if (x < 0) x += Lx;
    const bool own = lc >= RF_HALO && lc < RF_HALO + nout && strip * nout + lc - RF_HALO < Lx;
    const int cols[3] = {x == 0 ? Lx - 1 : x - 1, x, x == Lx - 1 ? 0 : x + 1};
    // segment rows [ys, ye); the top two rows always share one (the outflow
    // top adds to what row Ly - 2 stored, see stage P)
    const int ys = seg * seg_h;
    int ye = min(ys + seg_h, Ly);
    if (ye == Ly - 1) ye = Ly;
    if (ys >= Ly || (ys == Ly - 1 && ys > 0)) return;  // (the whole block: no barrier yet)
    const int cl = max(ys - 1, 0), ch = min(ye, Ly - 1);  // rows of stage C
    auto ring = [&](int f, int r) { return sm + (f * RF_R + (r & (RF_R - 1))) * RF_W + s; };
    const float G = P.G;

    float nr[5];  // ring inputs of one row (0 beyond the walls)
    auto load_ring = [&](int r, auto steady) {
        if (decltype(steady)::value || (r >= 0 && r < Ly)) {
            const int i = r * pitch + x;
            nr[0] = LB_LD(A.ldrx, i, pl);
            nr[1] = LB_LD(A.ldry, i, pl);
            nr[2] = LB_LD(A.ldivv, i, pl);
            nr[3] = LB_LD(A.lr_in, i, pl);
            nr[4] = LB_LD(A.psi, i, pl);
        } else {
            nr[0] = nr[1] = nr[2] = nr[3] = nr[4] = 0.f;
        }
    };
    auto store_ring = [&](int r) {
#pragma unroll
        for (int k = 0; k < 4; ++k) *ring(k, r) = nr[k];
        *ring(6, r) = nr[4];
    };
    // stage C's per-cell inputs of one row: pulled populations (Eq. 3; the
    // outflow top pulls 4, 7, 8 from its own row), lf part of lambda_f*^{n+1},
    // theta, and the thermal pass's lambda_v, lambda_rho, lambda_theta (psi
    // comes through its ring)
    float nf[9], nl[9], nlvx, nlvy, nlrho, nth, nlth;
    auto load_in = [&](int r, auto steady) {
        constexpr bool S = decltype(steady)::value;
        const int rc = r * pitch;
        const int rows[3] = {S || r > 0 ? rc - pitch : -1, rc,
                             S || r + 1 < Ly ? rc + pitch : (P.bc == BC_TOP_OUTFLOW ? rc : -1)};
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            const int rr = rows[1 - EYd[a]];
            nf[a] = !S && rr < 0 ? 0.f : LB_LD(A.fstar, a * pl + rr + cols[1 - EXd[a]], 9 * (size_t)pl);
        }
        const int i = rc + x;
#pragma unroll
        for (int a = 0; a < 9; ++a) nl[a] = LB_LD(A.lf_in, a * pl + i, 9 * (size_t)pl);
        nlvx = LB_LD(A.lvx, i, pl);
        nlvy = LB_LD(A.lvy, i, pl);
        nlrho = LB_LD(A.lrho, i, pl);
        nth = LB_LD(A.theta, i, pl);
        nlth = LB_LD(A.lth, i, pl);
    };
    // stage C's results for stage P, carried one iteration (row L - 1)
    float c_lrho = 0.f, c_lpsi = 0.f, c_psi = 0.f, c_rho = 0.f, c_th = 0.f, c_lth = 0.f;

    load_ring(cl - 1, std::false_type{});
    store_ring(cl - 1);
    load_ring(cl, std::false_type{});
    store_ring(cl);
    load_ring(cl + 1, std::false_type{});
    load_in(cl, std::false_type{});
    // one row iteration L; in a steady one (S) stage C's row is neither a
    // wall row nor the first fluid row and is the block's own, stage P's row
    // is the block's own, off the walls and above the heat-flux rows, and the
    // next rows' loads lie inside the grid, so those tests are compiled out
    auto iter = [&](const int L, auto steady) {
        constexpr bool S = decltype(steady)::value;
        // ---- ring row L + 1 and this row's inputs; then row L + 1's loads
        float f[9], lo[9];
        const float lvx_t = nlvx, lvy_t = nlvy, lrho_t = nlrho, th = nth;
        const float lth_t = nlth;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            f[a] = nf[a];
            lo[a] = nl[a];
        }
        if (S || L <= ch) store_ring(L + 1);
        if (S || L + 1 <= ch) {
            load_in(L + 1, steady);
            load_ring(L + 2, steady);
        }
        __syncthreads();

        // ---- C: row L
        float n_lrho = 0.f, n_lpsi = 0.f, n_rho = 0.f, n_psi = 0.f;
        if (S || L <= ch) {
            const int y = L;
            const bool wall = !S && (y == 0 || y == Ly - 1);
            wall_fill(P, y, f);
            // psi and F_m (Eq. 7) from the psi ring, as the step forms them; on
            // wall rows only with the ghost layer, whose row beyond the wall
            // is a copy of the wall row
            const float psi = ring(6, y)[0];
            float Fmx = 0.f, Fmy = 0.f;
            if (!wall || P.ghost) {
                const float* pc = ring(6, y);
                const float* pm = (wall && y == 0) ? pc : ring(6, y - 1);
                const float* pp = (wall && y == Ly - 1) ? pc : ring(6, y + 1);
                float sx, sy;  // 12 sum_a w_a psi(x + e_a) e_a
                grad12(pm, pc, pp, sx, sy);
                const float mG = -G * (1.f / 12.f) * psi;
                Fmx = mG * sx;
                Fmy = mG * sy;
            }
            float gx, gy, hx, hy, dvx, dvy;  // 12 D of ldrx, ldry, ldivv (gy, hx unused)
            grad12(ring(0, y - 1), ring(0, y), ring(0, y + 1), gx, gy);
            grad12(ring(1, y - 1), ring(1, y), ring(1, y + 1), hx, hy);
            grad12(ring(2, y - 1), ring(2, y), ring(2, y + 1), dvx, dvy);
            // lambda of f*^{n+1} here: lf part + lr of the cell that pulled it
#pragma unroll
            for (int a = 0; a < 9; ++a) lo[a] += ring(3, y + EYd[a])[EXd[a]];
            const float lr_c = -(gx + hy) * (1.f / 12.f);
            const float lvx_c = -dvx * (1.f / 12.f), lvy_c = -dvy * (1.f / 12.f);
            // rho, j, F, v of the step (Eqs. 6, 9, 22)
            const float rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
            const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
            const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
            const float Fx = Fmx;
            float Fy = Fmy;
            if (!wall) {
                if (!S && y == 1) Fy += P.gw6 * psi * psi;
                Fy -= P.g * (rho - P.rho_ave);
            }
            const float irho = rcp_a(rho);
            const float vx = (jx + 0.5f * Fx) * irho, vy = (jy + 0.5f * Fy) * irho;
            // lambda_dm = diag(1/9, 1/36, ...) M lambda_f*
            const float Ml1 = -4.f * lo[0] - (lo[1] + lo[2] + lo[3] + lo[4]) + 2.f * (lo[5] + lo[6] + lo[7] + lo[8]);
            const float Ml2 = 4.f * lo[0] - 2.f * (lo[1] + lo[2] + lo[3] + lo[4]) + (lo[5] + lo[6] + lo[7] + lo[8]);
            const float Ml3 = lo[1] - lo[3] + lo[5] - lo[6] - lo[7] + lo[8];
            const float Ml4 = -2.f * lo[1] + 2.f * lo[3] + lo[5] - lo[6] - lo[7] + lo[8];
            const float Ml5 = lo[2] - lo[4] + lo[5] + lo[6] - lo[7] - lo[8];
            const float Ml6 = -2.f * lo[2] + 2.f * lo[4] + lo[5] + lo[6] - lo[7] - lo[8];
            const float Ml7 = lo[1] - lo[2] + lo[3] - lo[4];
            const float Ml8 = lo[5] - lo[6] + lo[7] - lo[8];
            const float ldm1 = Ml1 * (1.f / 36.f), ldm2 = Ml2 * (1.f / 36.f), ldm3 = Ml3 * (1.f / 6.f);
            const float ldm4 = Ml4 * (1.f / 12.f), ldm5 = Ml5 * (1.f / 6.f), ldm6 = Ml6 * (1.f / 12.f);
            const float ldm7 = Ml7 * 0.25f, ldm8 = Ml8 * 0.25f;
            // forward quantities of dm
            const float v2 = vx * vx + vy * vy;
            const float m7 = f[1] - f[2] + f[3] - f[4];
            const float m8 = f[5] - f[6] + f[7] - f[8];
            const float ne7 = m7 - rho * (vx * vx - vy * vy);
            const float ne8 = m8 - rho * vx * vy;
            const float psi2 = psi * psi;
            const float ipsi2 = psi2 > 0.f ? rcp_a(psi2) : 0.f;
            const float R = (Fmx * Fmx + Fmy * Fmy) * ipsi2;
            const float S7 = 2.f * (vx * Fx - vy * Fy), S8 = vx * Fy + vy * Fx;
            const float sr = (rho - P.rho_v) * P.inv_drho;
            const float sfr = fminf(fmaxf(sr, 0.f), 1.f);
            const float snu = rcp_a(P.tau_v + P.dtau * sfr);
            // dm = -Lambda (m - meq) + (I - Lambda/2) S, momentum rows dm_j = F
            const float lne1 = -P.s_e * ldm1, lS1 = (1.f - 0.5f * P.s_e) * ldm1;
            const float lne2 = -P.s_z * ldm2, lS2 = (1.f - 0.5f * P.s_z) * ldm2;
            const float lne4 = -P.s_q * ldm4, lne6 = -P.s_q * ldm6;
            float lFx = ldm3 - (1.f - 0.5f * P.s_q) * ldm4;
            float lFy = ldm5 - (1.f - 0.5f * P.s_q) * ldm6;
            const float lne7 = -snu * ldm7, lS7 = (1.f - 0.5f * snu) * ldm7;
            const float lne8 = -snu * ldm8, lS8 = (1.f - 0.5f * snu) * ldm8;
            const float lsnu = -(ne7 + 0.5f * S7) * ldm7 - (ne8 + 0.5f * S8) * ldm8;
            // ne_k = m_k(f) - meq_k(rho, v): m part -> lambda_f = M^T lambda_m, plus
            // the identity part of f* = f + ...
            float lf[9];
            lf[0] = lo[0] - 4.f * lne1 + 4.f * lne2;
            lf[1] = lo[1] - lne1 - 2.f * lne2 - 2.f * lne4 + lne7;
            lf[2] = lo[2] - lne1 - 2.f * lne2 - 2.f * lne6 - lne7;
            lf[3] = lo[3] - lne1 - 2.f * lne2 + 2.f * lne4 + lne7;
            lf[4] = lo[4] - lne1 - 2.f * lne2 + 2.f * lne6 - lne7;
            lf[5] = lo[5] + 2.f * lne1 + lne2 + lne4 + lne6 + lne8;
            lf[6] = lo[6] + 2.f * lne1 + lne2 - lne4 + lne6 - lne8;
            lf[7] = lo[7] + 2.f * lne1 + lne2 - lne4 - lne6 + lne8;
            lf[8] = lo[8] + 2.f * lne1 + lne2 + lne4 - lne6 - lne8;
            // meq part (lambda_meq = -lambda_ne): meq1 = rho(-2 + 3v^2), meq2 = rho(1 - 3v^2),
            // meq4 = -rho vx, meq6 = -rho vy, meq7 = rho(vx^2 - vy^2), meq8 = rho vx vy
            const float q1 = -lne1, q2 = -lne2, q4 = -lne4, q6 = -lne6, q7 = -lne7, q8 = -lne8;
            float lrho = q1 * (-2.f + 3.f * v2) + q2 * (1.f - 3.f * v2) - q4 * vx - q6 * vy + q7 * (vx * vx - vy * vy) +
                         q8 * vx * vy;
            float lvx = q1 * 6.f * rho * vx - q2 * 6.f * rho * vx - q4 * rho + q7 * 2.f * rho * vx + q8 * rho * vy;
            float lvy = q1 * 6.f * rho * vy - q2 * 6.f * rho * vy - q6 * rho - q7 * 2.f * rho * vy + q8 * rho * vx;
            // S (Eq. 8): S1 = 6 vF + sig_e R, S2 = -6 vF - sig_z R, S7, S8
            const float lvF = 6.f * lS1 - 6.f * lS2;
            const float lR = P.sig_e * lS1 - P.sig_z * lS2;
            lvx += lvF * Fx + 2.f * lS7 * Fx + lS8 * Fy;
            lvy += lvF * Fy - 2.f * lS7 * Fy + lS8 * Fx;
            lFx += lvF * vx + 2.f * lS7 * vx + lS8 * vy;
            lFy += lvF * vy - 2.f * lS7 * vy + lS8 * vx;
            float lFmx = 0.f, lFmy = 0.f, lpsi = 0.f;
            if (psi2 > 0.f) {
                lFmx += 2.f * Fmx * lR * ipsi2;
                lFmy += 2.f * Fmy * lR * ipsi2;
                lpsi += -2.f * R * lR * psi * ipsi2;
            }
            // snu(rho)
            if (sr > 0.f && sr < 1.f) lrho += lsnu * (-snu * snu * P.dtau * P.inv_drho);
            // velocity v = (j + F/2) / rho with the thermal pass's lambda_v added
            lvx += lvx_t + lvx_c;
            lvy += lvy_t + lvy_c;
            lrho += lrho_t + lr_c;
            const float ljx = lvx * irho, ljy = lvy * irho;
            lFx += 0.5f * ljx;
            lFy += 0.5f * ljy;
            lrho += -(lvx * vx + lvy * vy) * irho;
#pragma unroll
            for (int a = 0; a < 9; ++a) lf[a] += EXd[a] * ljx + EYd[a] * ljy;
            // forces: F = F_m + F_ads + F_b on fluid rows; on wall rows F_m
            // with the ghost layer, else 0
            const bool mine = own && (S || (y >= ys && y < ye));
            if (!wall) {
                lFmx += lFx;
                lFmy += lFy;
                lrho += -P.g * lFy;  // F_b (Eq. 9)
                if (!S && y == 1) {  // F_ads (Eq. 22) on the first fluid row
                    lpsi += 2.f * P.gw6 * psi * lFy;
                    if (mine) LB_ADD(A.dGwx, x, P.pitch, (double)(psi2 * (1.f / 6.f) * lFy));  // one cell per x on this row
                }
                if (psi > 0.f) lpsi += (Fmx * lFmx + Fmy * lFmy) * rcp_a(psi);  // own factor of F_m
            } else if (P.ghost) {
                lFmx += lFx;
                lFmy += lFy;
                if (psi > 0.f) lpsi += (Fmx * lFmx + Fmy * lFmy) * rcp_a(psi);
            } else {
                lFmx = lFmy = 0.f;  // no force is applied on wall rows
            }
            *ring(4, y) = psi * lFmx;
            *ring(5, y) = psi * lFmy;
            if (mine) {
                if (wall) {  // the wall row's lambda, completed by stage P
                    const int o = (y == 0 ? 0 : pitch) + x;
#pragma unroll
                    for (int a = 0; a < 9; ++a) LB_ST(A.sb, o + 2 * a * pitch, 18 * (size_t)pitch, lf[a]);
                } else {  // pull-streaming transposed: lambda of f*_a(y - e_a) (always inside)
#pragma unroll
                    for (int a = 0; a < 9; ++a)
                        LB_ST(A.lf_out, a * pl + (y - EYd[a]) * pitch + cols[1 - EXd[a]], 9 * (size_t)pl, lf[a]);
                }
            }
            n_lrho = lrho;
            n_lpsi = lpsi;
            n_rho = rho;
            n_psi = psi;
        }
        __syncthreads();

        // ---- P: row L - 1
        const int r = L - 1;
        if ((S || (r >= ys && r < ye)) && own) {
            const bool wall = !S && (r == 0 || r == Ly - 1);
            const int i = r * pitch + x;
            // F_m's neighbour sums transposed: lambda_psi += G (Dx[Qx] + Dy[Qy]);
            // rows beyond the walls hold no cell
            const float* xm = ring(4, r - 1);
            const float* xc = ring(4, r);
            const float* xp = ring(4, r + 1);
            const float* ym = ring(5, r - 1);
            const float* yp = ring(5, r + 1);
            float dq = 4.f * (xc[1] - xc[-1]);
            if (S || r > 0) dq += (xm[1] - xm[-1]) - (4.f * ym[0] + ym[1] + ym[-1]);
            if (S || r + 1 < Ly) dq += (xp[1] - xp[-1]) + (4.f * yp[0] + yp[1] + yp[-1]);
            if (!S && P.ghost && wall) {
                // the ghost row beyond this wall row is a copy of it: the
                // row's cells that reached across the wall read psi here
                // too (bottom: through e_y = -1, top: e_y = +1)
                const float* yc = ring(5, r);
                const float g = 4.f * yc[0] + yc[1] + yc[-1];
                dq += (xc[1] - xc[-1]) + (r == 0 ? g : -g);
            }
            const float lpsi = c_lpsi + G * (1.f / 12.f) * dq;
            float lrho = c_lrho, lth = c_lth;
            if (c_psi > 0.f) {  // psi^2 = 2 (p_EOS - rho/3) / G (Eq. 21)
                const Eos e = eos(c_rho, P.Ts + c_th, P);
                const float k = lpsi * rcp_a(G * c_psi);
                lrho += k * (e.p_rho - 1.f / 3.f);
                lth += k * e.p_T;
            }
            // q(t) = (1/Lx) sum_x -cvchi rho(x,0) (-3 th0 + 4 th1 - th2) / 2 (Sec. 3.2)
            if (!S && lq != 0.f && r <= 2) {
                const float c = lq / (float)Lx * (-P.cvchi);
                const float rho0 = r == 0 ? c_rho : LB_LD(A.rho, x, pl);
                if (r == 0) {
                    lrho += c * 0.5f * (-3.f * c_th + 4.f * LB_LD(A.theta, pitch + x, pl) - LB_LD(A.theta, 2 * pitch + x, pl));
                    lth += c * rho0 * (-1.5f);
                } else if (r == 1) {
                    lth += c * rho0 * 2.f;
                } else {
                    lth += c * rho0 * (-0.5f);
                }
            }
            LB_ST(A.lt_out, i, pl, lth);
            if (!wall) {
                LB_ST(A.lr_out, i, pl, lrho);
            } else {
                LB_ST(A.lr_out, i, pl, 0.f);
                float lf[9];
                const int o = (r == 0 ? 0 : pitch) + x;
#pragma unroll
                for (int a = 0; a < 9; ++a) lf[a] = LB_LD(A.sb, o + 2 * a * pitch, 18 * (size_t)pitch) + lrho;
                // Zou-He fill transposed: the filled populations pass their
                // adjoint to the known ones they were built from
                if (r == 0) {
                    lf[4] += lf[2];
                    lf[7] += lf[5];
                    lf[1] += -0.5f * lf[5] + 0.5f * lf[6];
                    lf[3] += 0.5f * lf[5] - 0.5f * lf[6];
                    lf[8] += lf[6];
                    lf[2] = lf[5] = lf[6] = 0.f;
                } else if (P.bc == BC_WALLS) {
                    lf[2] += lf[4];
                    lf[5] += lf[7];
                    lf[1] += 0.5f * lf[7] - 0.5f * lf[8];
                    lf[3] += -0.5f * lf[7] + 0.5f * lf[8];
                    lf[6] += lf[8];
                    lf[4] = lf[7] = lf[8] = 0.f;
                }
                // pull-streaming transposed as a scatter; where y + e_a lies
                // beyond the wall f*_a of this cell has no consumer: 0
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int t = r - EYd[a];
                    if (t >= 0 && t < Ly) LB_ST(A.lf_out, a * pl + t * pitch + cols[1 - EXd[a]], 9 * (size_t)pl, lf[a]);
                    const int u = r + EYd[a];
                    if (u < 0 || u >= Ly) LB_ST(A.lf_out, a * pl + i, 9 * (size_t)pl, 0.f);
                }
                // the outflow top pulled populations 4, 7, 8 from its own row:
                // f*_a(x - e_a, Ly - 1) has this second consumer besides the
                // cell one row down, which is this thread's column too and
                // stored its share in stage C two rows ago
                if (P.bc == BC_TOP_OUTFLOW && r == Ly - 1) {
                    const int row = r * pitch;
                    LB_ADD(A.lf_out, 4 * pl + row + x, 9 * (size_t)pl, lf[4]);
                    LB_ADD(A.lf_out, 7 * pl + row + cols[2], 9 * (size_t)pl, lf[7]);
                    LB_ADD(A.lf_out, 8 * pl + row + cols[0], 9 * (size_t)pl, lf[8]);
                }
            }
        }
        c_lrho = n_lrho;
        c_lpsi = n_lpsi;
        c_rho = n_rho;
        c_psi = n_psi;
        c_th = th;
        c_lth = lth_t;
    };
    // steady iterations: stage C's row L in [max(ys, 2), min(ye, Ly - 2)),
    // stage P's row L - 1 in [max(ys, 3), ye), the next rows' loads
    // (L + 1 <= ch, L + 2 <= Ly - 1) inside
    const int Ls = max(ys + 1, 4);
    const int Le = min(min(ch - 1, Ly - 3), ye - 1) + 1;
    int L = cl;
    for (; L < Ls; ++L) iter(L, std::false_type{});
    for (; L < Le; ++L) iter(L, std::true_type{});
    for (; L <= ch + 1; ++L) iter(L, std::false_type{});
}

// Work-buffer layout: 7 field planes, the wall rows' lambda of the pulled
// populations [9][2][pitch], then dJ/d theta_b [pitch doubles], the
// per-column dJ/dG_w parts [pitch doubles] and dJ/dG_w.
constexpr int kPlanes = 7;
inline size_t sb_floats(const StepParams& P) { return 18 * (size_t)P.pitch; }

AdjFields fields_at(const StepParams& P, void* work) {
    float* w = (float*)work;
    const size_t pl = (size_t)P.plane;
    size_t k = 0;
    auto next = [&](int n) {
        float* p = w + k * pl;
        k += n;
        return p;
    };
    AdjFields A;
    A.fstar = nullptr;
    A.theta = nullptr;
    A.lf_in = A.lt_in = A.lr_in = nullptr;
    A.lf_out = A.lt_out = A.lr_out = nullptr;
    A.rho = A.psi = nullptr;
    A.drx = A.dry = A.divv = A.ax = A.ay = A.u2 = A.u3 = A.u4 = nullptr;
    A.lrho = next(1);
    A.lvx = next(1);
    A.lvy = next(1);
    A.lth = next(1);
    A.ldrx = next(1);
    A.ldry = next(1);
    A.ldivv = next(1);
    A.sb = w + kPlanes * pl;
    A.dTb = (double*)(A.sb + sb_floats(P));
    A.dGwx = A.dTb + P.pitch;
    A.dGw = A.dGwx + P.pitch;
    return A;
}

// dGw = sum over x of dGwx (one block, fixed order: reproducible)
__global__ void sum_columns(const double* __restrict__ v, int n, double* out) {
    __shared__ double part[256];
    double s = 0.0;
    for (int x = threadIdx.x; x < n; x += 256) s += v[x];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

__global__ void add_wall_row(const StepParams P, const float* lt, double* dTb) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < P.Lx) dTb[x] += (double)lt[x];
}

}  // namespace

size_t adjoint_work_bytes(const StepParams& P) {
    return sizeof(float) * ((size_t)kPlanes * (size_t)P.plane + sb_floats(P)) +
           sizeof(double) * (2 * (size_t)P.pitch + 2);
}

cudaError_t adjoint_grads_reset(const StepParams& P, void* work, cudaStream_t st) {
    AdjFields A = fields_at(P, work);
    return cudaMemsetAsync(A.dTb, 0, sizeof(double) * (2 * (size_t)P.pitch + 1), st);
}

cudaError_t adjoint_grads_finish(const StepParams& P, void* work, const float* lt0, double* dTb_host,
                                 double* dGw_host, cudaStream_t st) {
    AdjFields A = fields_at(P, work);
    if (P.bc != BC_PERIODIC) add_wall_row<<<(P.Lx + 127) / 128, 128, 0, st>>>(P, lt0, A.dTb);
    sum_columns<<<1, 256, 0, st>>>(A.dGwx, P.Lx, A.dGw);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && dTb_host)
        e = cudaMemcpyAsync(dTb_host, A.dTb, sizeof(double) * P.Lx, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && dGw_host) e = cudaMemcpyAsync(dGw_host, A.dGw, sizeof(double), cudaMemcpyDeviceToHost, st);
    return e;
}

// One reverse step: state (fstar, theta) of level n and the intermediates R
// of the step from it, lambda of level n+1 in (lf_in with lr_in, lt_in),
// lambda of level n out (lf_out with lr_out, lt_out); lq = dJ/dq(t_n). L is a dual-strip
// launch shape matching P (nout, nstrips, seg_h) for the recompute.
cudaError_t adjoint_reverse_step(const StepParams& P, const RecomputeOut& R, void* work, const float* fstar,
                                 const float* theta, const float* lf_in, const float* lt_in, const float* lr_in,
                                 float* lf_out, float* lt_out, float* lr_out, float lq, cudaStream_t st) {
    AdjFields A = fields_at(P, work);
    A.fstar = fstar;
    A.theta = theta;
    A.lf_in = lf_in;
    A.lt_in = lt_in;
    A.lr_in = lr_in;
    A.lf_out = lf_out;
    A.lt_out = lt_out;
    A.lr_out = lr_out;
    A.rho = R.rho;
    A.psi = R.psi;
    A.drx = R.drx;
    A.dry = R.dry;
    A.divv = R.divv;
    A.ax = R.ax;
    A.ay = R.ay;
    A.u2 = R.u2;
    A.u3 = R.u3;
    A.u4 = R.u4;
    // the four RK stages transposed, then the collision, forces, psi and the
    // pull: two column-marching launches, segments sized so that the blocks
    // fill the GPU once
    // SM count and blocks per SM of the two reverse kernels: looked up once
    // (a function-local static: initialised once, also under concurrent
    // first calls)
    struct RevShape {
        cudaError_t e;
        int nsm, occ_t, occ_f;
    };
    static const RevShape RS = [] {
        RevShape r{cudaSuccess, 0, 0, 0};
        int dev = 0;
        r.e = cudaGetDevice(&dev);
        if (r.e == cudaSuccess) r.e = cudaDeviceGetAttribute(&r.nsm, cudaDevAttrMultiProcessorCount, dev);
        if (r.e == cudaSuccess)
            r.e = cudaFuncSetAttribute(rev_thermal_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)rt_smem_bytes());
        if (r.e == cudaSuccess)
            r.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ_t, rev_thermal_fused, RT_BD, rt_smem_bytes());
        if (r.e == cudaSuccess) r.e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.occ_f, rev_flow_fused, RF_BD, 0);
        r.occ_t = std::max(r.occ_t, 1);
        r.occ_f = std::max(r.occ_f, 1);
        return r;
    }();
    if (RS.e != cudaSuccess) return RS.e;
    const int nsm = RS.nsm, occ_t = RS.occ_t, occ_f = RS.occ_f;
    // (a floor of 4 rows per segment: on small domains more, shorter marches
    // beat fewer long ones despite the halo rows; measured cost of the 256^2,
    // 2000-step adjoint against its forward steps: 2.78x at 4, 2.90x at 1,
    // 3.11x at 8, 4.06x at 16; at 512^2: 3.48x, 3.67x, 3.60x, 4.27x)
    auto shape = [&](int nout, int occ, int& seg_h) {  // -> number of blocks
        const int nstrips = (P.Lx + nout - 1) / nout;
        const int nseg = std::max(1, nsm * occ / nstrips);
        seg_h = std::max(4, (P.Ly + nseg - 1) / nseg);
        return nstrips * ((P.Ly + seg_h - 1) / seg_h);
    };
    int seg_t = 0, seg_f = 0;
    const int nb_t = shape(RT_BD - 2 * RT_HALO, occ_t, seg_t);
    rev_thermal_fused<<<nb_t, RT_BD, rt_smem_bytes(), st>>>(P, A, seg_t);
    const int nb_f = shape(RF_BD - 2 * RF_HALO, occ_f, seg_f);
    rev_flow_fused<<<nb_f, RF_BD, 0, st>>>(P, A, lq, seg_f);
    return cudaGetLastError();
}

}  // namespace lbgpu
