// Discrete adjoint of one time step (reverse mode), for gradients of the
// time-averaged bottom-wall heat flux J = (1/S) sum_n q(t_n) (Sec. 3.2) with
// respect to the wall temperature profile T_b(x) and the wettability G_w of
// Eq. 22.
//
// Forward intermediates of step n are recomputed from the stored state
// (f*^n, theta^n): on large domains by the fused step itself in its
// recompute mode (lb_step3.cu, RecomputeOut), on small ones by field kernels
// (one thread per cell) that follow its formulas. The reverse passes then
// transpose each part of the step in the opposite order:
//
//   RK4 of Eq. 18 (stage 4 .. 1)   -> lambda_theta, lambda of the per-cell
//   and the coefficients              coefficients (ax, ay, cA, cB), then
//   (rev_thermal_fused: one           lambda_rho, lambda_v through grad rho
//   column-marching launch)           and div v
//   MRT collision (Eqs. 2, 5, 8), v (Eq. 6), forces (Eqs. 7, 9, 22)
//                                  -> lambda_f, lambda_rho, lambda_psi, lambda_F_m
//   F_m neighbour sums (Eq. 7), psi (Eq. 21), q_w, rho = sum f
//                                  -> lambda_f, lambda_theta
//   Zou-He fill, pull-streaming (Eq. 3)
//                                  -> lambda_f*^n
//
// A stencil applied forward as out(x) = sum_d c_d in(x + d) is transposed as
// a gather lambda_in(y) += sum_d c_d lambda_out(y - d). Fields are pitched
// [Ly][pitch] FP32; gradients are accumulated in FP64. Supported: walls in
// y or the outflow top, no ghost layer (the host checks).
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

// stencil weights for offset (dx, dy): first derivatives (Lee and Lin) and
// the Laplacian; the first-derivative weights are also Eq. 7's w_a e_a.
__device__ __forceinline__ float wdx(int dx, int dy) {
    return dx == 0 ? 0.f : (dy == 0 ? dx * (1.f / 3.f) : dx * (1.f / 12.f));
}
__device__ __forceinline__ float wdy(int dx, int dy) {
    return dy == 0 ? 0.f : (dx == 0 ? dy * (1.f / 3.f) : dy * (1.f / 12.f));
}
__device__ __forceinline__ float wlap(int dx, int dy) {
    return (dx == 0 && dy == 0) ? (-20.f / 6.f) : ((dx == 0 || dy == 0) ? (4.f / 6.f) : (1.f / 6.f));
}

struct Grid {
    int Lx, Ly, pitch, bc;
    // index of (x + dx, y + dy) or -1 outside a wall-bounded domain
    __device__ __forceinline__ int at(int x, int y, int dx, int dy) const {
        int xx = x + dx;
        if (xx < 0) xx += Lx;
        if (xx >= Lx) xx -= Lx;
        int yy = y + dy;
        if (bc == BC_PERIODIC) {
            if (yy < 0) yy += Ly;
            if (yy >= Ly) yy -= Ly;
        } else if (yy < 0 || yy >= Ly) {
            return -1;
        }
        return yy * pitch + xx;
    }
    __device__ __forceinline__ bool wall(int y) const { return bc != BC_PERIODIC && (y == 0 || y == Ly - 1); }
};

// All the field planes one adjoint step works on.
struct AdjFields {
    // forward intermediates of the step being reversed
    const float* fstar;  // f*^n, 9 planes
    const float* theta;  // theta^n
    float *rho, *psi, *jx, *jy, *Fmx, *Fmy, *Fx, *Fy, *vx, *vy;
    float *drx, *dry, *divv, *ax, *ay, *cA, *cB;
    float *u2, *u3, *u4;
    // adjoints
    const float* lf_in;  // lambda of f*^{n+1}, 9 planes
    const float* lt_in;  // lambda of theta^{n+1}
    float* lf_out;       // lambda of f*^n, 9 planes
    float* lt_out;       // lambda of theta^n
    float* lf;           // lambda of the pulled populations, 9 planes
    float *lrho, *lpsi, *lFmx, *lFmy, *lvx, *lvy, *lth;
    float *ldrx, *ldry, *ldivv;
    double* dTb;   // [Lx] dJ/d theta_b accumulators
    double* dGwx;  // [Lx] dJ/dG_w contributions of each column's first fluid row
    double* dGw;   // dJ/dG_w (sum of dGwx, formed at the end)
};

__device__ __forceinline__ bool cell(const StepParams& P, int& x, int& y, int& i) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    i = y * P.pitch + x;
    return x < P.Lx && y < P.Ly;
}

__device__ __forceinline__ Grid grid_of(const StepParams& P) { return Grid{P.Lx, P.Ly, P.pitch, P.bc}; }

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

// Pulled and wall-filled populations of cell (x, y) from f* (Eq. 3, Zou-He
// on the wall rows), as the step computes them.
__device__ __forceinline__ void pull_cell(const StepParams& P, const float* __restrict__ fstar, int x, int y,
                                          float (&f)[9]) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        int yy = y - EYd[a];
        bool ok = true;
        if (P.bc == BC_PERIODIC) {
            if (yy < 0) yy += P.Ly;
            if (yy >= P.Ly) yy -= P.Ly;
        } else {
            // the outflow top pulls its unknowns from the top row itself
            if (P.bc == BC_TOP_OUTFLOW && yy == P.Ly) yy = P.Ly - 1;
            ok = yy >= 0 && yy < P.Ly;
        }
        int xx = x - EXd[a];
        if (xx < 0) xx += P.Lx;
        if (xx >= P.Lx) xx -= P.Lx;
        f[a] = ok ? fstar[a * P.plane + yy * P.pitch + xx] : 0.f;
    }
    wall_fill(P, y, f);
}

// ---- forward recompute by field kernels ---------------------------------------
//
// For small domains, where the fused step's 5-row pipeline halo and its
// sequential march dominate (a 256 x 256 step takes ~20 us in it), the
// intermediates are recomputed by these one-thread-per-cell kernels, which
// follow the fused step's formulas.

__global__ void fwd_pull(const StepParams P, AdjFields A) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    float f[9];
    pull_cell(P, A.fstar, x, y, f);
    float rho = 0.f;
    for (int a = 0; a < 9; ++a) rho += f[a];
    A.rho[i] = rho;
    A.jx[i] = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    A.jy[i] = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    const float T = P.Ts + A.theta[i];
    const float arg = P.two_over_G * (eos(rho, T, P).p - rho * (1.f / 3.f));
    A.psi[i] = arg > 0.f ? sqrtf(arg) : 0.f;
    (void)g;
}

__global__ void fwd_force(const StepParams P, AdjFields A) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    const bool wall = g.wall(y);
    float Fmx = 0.f, Fmy = 0.f;
    if (!wall) {
        float sx = 0.f, sy = 0.f;
        for (int a = 1; a < 9; ++a) {
            const float pn = A.psi[g.at(x, y, EXd[a], EYd[a])];
            sx += wdx(EXd[a], EYd[a]) * pn;
            sy += wdy(EXd[a], EYd[a]) * pn;
        }
        Fmx = -P.G * A.psi[i] * sx;
        Fmy = -P.G * A.psi[i] * sy;
    }
    float Fx = Fmx, Fy = Fmy;
    if (!wall) {
        if (P.bc != BC_PERIODIC && y == 1) Fy += P.gw6 * A.psi[i] * A.psi[i];
        Fy -= P.g * (A.rho[i] - P.rho_ave);
    }
    A.Fmx[i] = Fmx;
    A.Fmy[i] = Fmy;
    A.Fx[i] = Fx;
    A.Fy[i] = Fy;
    A.vx[i] = (A.jx[i] + 0.5f * Fx) / A.rho[i];
    A.vy[i] = (A.jy[i] + 0.5f * Fy) / A.rho[i];
}

__global__ void fwd_coef(const StepParams P, AdjFields A) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    if (g.wall(y)) {
        A.drx[i] = A.dry[i] = A.divv[i] = A.ax[i] = A.ay[i] = A.cA[i] = A.cB[i] = 0.f;
        return;
    }
    float drx = 0.f, dry = 0.f, dvx = 0.f, dvy = 0.f;
    for (int a = 1; a < 9; ++a) {
        const int j = g.at(x, y, EXd[a], EYd[a]);
        const float cx = wdx(EXd[a], EYd[a]), cy = wdy(EXd[a], EYd[a]);
        drx += cx * A.rho[j];
        dry += cy * A.rho[j];
        dvx += cx * A.vx[j];
        dvy += cy * A.vy[j];
    }
    const float rho = A.rho[i];
    const float divv = dvx + dvy;
    const float br = P.b * rho;
    A.drx[i] = drx;
    A.dry[i] = dry;
    A.divv[i] = divv;
    A.ax[i] = -A.vx[i] + P.chi * drx / rho;
    A.ay[i] = -A.vy[i] + P.chi * dry / rho;
    A.cA[i] = divv * P.R * P.inv_cv / (1.f - br);
    A.cB[i] = divv * P.a * rho * P.inv_cv / (1.f + 2.f * br - br * br);
}

// u_out = theta + c K(u_in) on fluid rows, theta on wall rows (Eqs. 18-20).
__global__ void fwd_stage(const StepParams P, AdjFields A, const float* u_in, float* u_out, float c) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    const bool wall = g.wall(y);
    if (wall) {
        u_out[i] = A.theta[i];
        return;
    }
    float dx = 0.f, dy = 0.f, lap = wlap(0, 0) * u_in[i];
    for (int a = 1; a < 9; ++a) {
        const float un = u_in[g.at(x, y, EXd[a], EYd[a])];
        dx += wdx(EXd[a], EYd[a]) * un;
        dy += wdy(EXd[a], EYd[a]) * un;
        lap += wlap(EXd[a], EYd[a]) * un;
    }
    const float T = P.Ts + u_in[i];
    const float dphi = P.k1k1 - P.k0k1 / sqrtf(T);
    const float K = A.ax[i] * dx + A.ay[i] * dy + P.chi * lap - T * (A.cA[i] - A.cB[i] * dphi);
    u_out[i] = A.theta[i] + c * K;
}

// ---- reverse -----------------------------------------------------------------

// coefficients -> lambda of grad rho, div v (local) and the local parts of
// lambda_rho, lambda_v, for cell i (after the last stage's accumulation)
__device__ __forceinline__ void rev_coef_vals(const StepParams& P, const AdjFields& A, int i, bool wall, float lax,
                                              float lay, float lcA, float lcB) {
    if (wall) {
        A.ldrx[i] = A.ldry[i] = A.ldivv[i] = 0.f;
        A.lrho[i] = A.lvx[i] = A.lvy[i] = 0.f;
        return;
    }
    const float rho = A.rho[i], irho = rcp_a(rho);
    const float br = P.b * rho;
    const float i1 = rcp_a(1.f - br);
    const float D = 1.f + 2.f * br - br * br, iD = rcp_a(D);
    const float dD = 2.f * P.b - 2.f * P.b * br;
    const float divv = A.divv[i];
    A.ldrx[i] = P.chi * lax * irho;
    A.ldry[i] = P.chi * lay * irho;
    A.ldivv[i] = lcA * P.R * P.inv_cv * i1 + lcB * P.a * rho * P.inv_cv * iD;
    A.lrho[i] = -P.chi * (A.drx[i] * lax + A.dry[i] * lay) * irho * irho + lcA * divv * P.R * P.inv_cv * P.b * i1 * i1 +
                lcB * divv * P.a * P.inv_cv * (D - rho * dD) * iD * iD;
    A.lvx[i] = -lax;
    A.lvy[i] = -lay;
}

// ---- the four RK stages transposed in one column-marching launch ------------
//
// Each RK stage of Eq. 18 (stage 4 .. 1) transposed and then the
// coefficients (rev_coef_vals), cell by cell, in one pass over the domain: a
// block of RT_BD threads owns RT_BD - 2 RT_HALO output columns and a segment
// of rows and marches up the segment one row per iteration, each thread one
// column:
//
//   S  row L    : mu4 = lambda_theta'/6 (fluid rows) and its products with
//                 ax, ay into shared rings; u4, u3 (row L), u2 (row L - 2),
//                 theta (row L - 3); ax, ay, cA, cB, lambda-bar (own column)
//   R4 row L-1  : stage 4 transposed (rows L-2..L) -> mu3 and its products
//   R3 row L-2  : stage 3 transposed -> mu2
//   R2 row L-3  : stage 2 transposed -> mu1
//   R1 row L-4  : stage 1 transposed; the cell's coefficient adjoints are
//                 complete: lambda of grad rho, div v, rho, v, theta out
//
// A stage's lambda_u at x gathers c_d(x - d) mu(x - d) over the 9 cells
// around x, with c_d(s) = ax(s) wx(d) + ay(s) wy(d) + chi wl(d) the
// isotropic stencils of Sec. 2. With the products PX = ax mu and PY = ay mu
// stored at the source cell, and the first-derivative weights odd in d,
// that is lambda_u = -Dx[PX] - Dy[PY] + chi Lap[mu]: the forward stencils
// applied to the products. Each stage reaches one column further out: 4
// halo columns per side. The per-cell accumulators (coefficient adjoints,
// lambda_theta) ride along with their row in registers. Walls in y only
// (the adjoint's supported case). (Measured: this scalar form with 4 warps
// per block runs 1.5 x faster than a paired-FP32 form over two strips,
// whose shared rings allowed only 10 warps per SM.)
constexpr int RT_BD = 128, RT_HALO = 4, RT_W = RT_BD + 2, RT_R = 4;  // ring rows

__global__ void __launch_bounds__(RT_BD) rev_thermal_fused(const StepParams P, AdjFields A, int seg_h) {
    extern __shared__ float rt_sm[];
    float* const sPX = rt_sm;                   // per stage (4, 3, 2, 1 -> 0..3): [4][RT_R][RT_W]
    float* const sPY = sPX + 4 * RT_R * RT_W;
    float* const sMU = sPY + 4 * RT_R * RT_W;
    float* const sU = sMU + 4 * RT_R * RT_W;    // u4, u3, u2, theta: [4][RT_R][RT_W]
    float* const sOWN = sU + 4 * RT_R * RT_W;   // ax, ay, cA, cB, lambda-bar: [5][RT_R][RT_BD]
    constexpr int SMN = 16 * RT_R * RT_W + 5 * RT_R * RT_BD;
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
    auto own = [&](int f, int r) -> float& { return sOWN[(f * RT_R + (r & (RT_R - 1))) * RT_BD + lc]; };
    auto ring = [&](float* base, int k, int r) { return base + (k * RT_R + (r & (RT_R - 1))) * RT_W + s; };
    float acc_ax[4], acc_ay[4], acc_cA[4], acc_cB[4], acc_th[4];  // index k: the row stage k worked on
#pragma unroll
    for (int k = 0; k < 4; ++k) acc_ax[k] = acc_ay[k] = acc_cA[k] = acc_cB[k] = acc_th[k] = 0.f;
    __syncthreads();

    // stage k (0: stage 4 .. 3: stage 1) at row r
    auto stage = [&](const int k, const int r) {
        const bool wall = r == 0 || r == Ly - 1;
        // rows beyond the walls hold no cell: their products are 0
        const bool hm = r - 1 >= 0, hp = r + 1 < Ly;
        const float* xm = ring(sPX, k, r - 1);
        const float* xc = ring(sPX, k, r);
        const float* xp = ring(sPX, k, r + 1);
        const float* ym = ring(sPY, k, r - 1);
        const float* yp = ring(sPY, k, r + 1);
        const float* mm = ring(sMU, k, r - 1);
        const float* mc = ring(sMU, k, r);
        const float* mp = ring(sMU, k, r + 1);
        // 12 Dx[PX], 12 Dy[PY], 6 Lap[mu] (unweighted sums of the stencils)
        float dxp = 4.f * (xc[1] - xc[-1]), dyp = 0.f;
        float lap = -20.f * mc[0] + 4.f * (mc[1] + mc[-1]);
        if (hm) {
            dxp += xm[1] - xm[-1];
            dyp -= 4.f * ym[0] + ym[1] + ym[-1];
            lap += 4.f * mm[0] + mm[1] + mm[-1];
        }
        if (hp) {
            dxp += xp[1] - xp[-1];
            dyp += 4.f * yp[0] + yp[1] + yp[-1];
            lap += 4.f * mp[0] + mp[1] + mp[-1];
        }
        float lu = -(dxp + dyp) * (1.f / 12.f) + chi * (1.f / 6.f) * lap;
        const float m = mc[0];
        float lax = 0.f, lay = 0.f, lcA = 0.f, lcB = 0.f;
        if (!wall && m != 0.f) {
            const float* um = ring(sU, k, r - 1);
            const float* uc = ring(sU, k, r);
            const float* up = ring(sU, k, r + 1);
            const float T = P.Ts + uc[0];
            const float rsq = rsqrt_a(T);
            const float dphi = P.k1k1 - P.k0k1 * rsq;
            const float d2phi = 0.5f * P.k0k1 * (rsq * rsq * rsq);
            const float cA = own(2, r), cB = own(3, r);
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
            acc_th[0] = own(4, r) + lu;
        } else {
            acc_ax[k] += lax;
            acc_ay[k] += lay;
            acc_cA[k] += lcA;
            acc_cB[k] += lcB;
            acc_th[k] += lu;
        }
        if (k < 3) {  // the next stage's mu = a lambda-bar + b lambda_u on fluid rows, with its products
            const float ab = k == 2 ? 1.f / 6.f : 1.f / 3.f, bb = k == 0 ? 1.f : 0.5f;
            const float mn = wall ? 0.f : ab * own(4, r) + bb * lu;
            *ring(sMU, k + 1, r) = mn;
            *ring(sPX, k + 1, r) = own(0, r) * mn;
            *ring(sPY, k + 1, r) = own(1, r) * mn;
        }
    };

    // the inputs of iteration L, loaded one iteration ahead (their latency is
    // hidden behind the stages): lambda_theta', ax, ay, u4, u3 of row L, cA,
    // cB of row L - 1, u2 of row L - 2, theta of row L - 3
    float n_lin = 0.f, n_ax = 0.f, n_ay = 0.f, n_u4 = 0.f, n_u3 = 0.f, n_cA = 0.f, n_cB = 0.f, n_u2 = 0.f, n_th = 0.f;
    auto prefetch = [&](int L) {
        if (L <= hi) {
            const int i = L * pitch + x;
            n_lin = A.lt_in[i];
            n_ax = A.ax[i];
            n_ay = A.ay[i];
            n_u4 = A.u4[i];
            n_u3 = A.u3[i];
        }
        if (L - 1 >= lo && L - 1 <= hi) {
            const int i = (L - 1) * pitch + x;
            n_cA = A.cA[i];
            n_cB = A.cB[i];
        }
        if (L - 2 >= lo && L - 2 <= hi) n_u2 = A.u2[(L - 2) * pitch + x];
        if (L - 3 >= lo && L - 3 <= hi) n_th = A.theta[(L - 3) * pitch + x];
    };
    prefetch(lo);
    for (int L = lo; L <= hi + RT_HALO; ++L) {
        // ---- S: the prefetched row into the rings, then the next one's loads
        if (L <= hi) {
            const bool wall = L == 0 || L == Ly - 1;
            const float mu = wall ? 0.f : n_lin * (1.f / 6.f);
            *ring(sMU, 0, L) = mu;
            *ring(sPX, 0, L) = n_ax * mu;
            *ring(sPY, 0, L) = n_ay * mu;
            own(0, L) = n_ax;
            own(1, L) = n_ay;
            own(4, L) = wall ? 0.f : n_lin;
            *ring(sU, 0, L) = n_u4;
            *ring(sU, 1, L) = n_u3;
        }
        if (L - 1 >= lo && L - 1 <= hi) {  // cA, cB of row L - 1 (stage 4 there next)
            own(2, L - 1) = n_cA;
            own(3, L - 1) = n_cB;
        }
        if (L - 2 >= lo && L - 2 <= hi) *ring(sU, 2, L - 2) = n_u2;
        if (L - 3 >= lo && L - 3 <= hi) *ring(sU, 3, L - 3) = n_th;
        prefetch(L + 1);
        __syncthreads();
        if (L - 1 >= lo && L - 1 <= hi) stage(0, L - 1);
        __syncthreads();
        if (L - 2 >= lo && L - 2 <= hi) stage(1, L - 2);
        __syncthreads();
        if (L - 3 >= lo && L - 3 <= hi) stage(2, L - 3);
        __syncthreads();
        const int r = L - 4;
        if (r >= ys && r < ye) {
            stage(3, r);
            if (out) {
                const int i = r * pitch + x;
                A.lth[i] = acc_th[3];
                rev_coef_vals(P, A, i, r == 0 || r == Ly - 1, acc_ax[3], acc_ay[3], acc_cA[3], acc_cB[3]);
                if (r == 0) A.dTb[x] += (double)A.lt_in[i];
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
    }
}

constexpr size_t rt_smem_bytes() { return sizeof(float) * (16 * (size_t)RT_R * RT_W + 5 * (size_t)RT_R * RT_BD); }

// MRT collision (additive form f* = f + M^-1 dm), velocity and the local
// parts of the forces, transposed cell by cell; first the transposed
// gradients of the RK coefficients (lambda_rho += Dx^T ldrx + Dy^T ldry,
// lambda_v += D^T ldivv), which complete this cell's lambda_rho and lambda_v.
__global__ void rev_collide(const StepParams P, AdjFields A) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    const bool wall = g.wall(y);
    float lr_c = 0.f, lvx_c = 0.f, lvy_c = 0.f;
    for (int a = 1; a < 9; ++a) {
        const int j = g.at(x, y, -EXd[a], -EYd[a]);
        if (j < 0) continue;
        const float cx = wdx(EXd[a], EYd[a]), cy = wdy(EXd[a], EYd[a]);
        lr_c += cx * A.ldrx[j] + cy * A.ldry[j];
        lvx_c += cx * A.ldivv[j];
        lvy_c += cy * A.ldivv[j];
    }
    const int pl = P.plane;
    float f[9], lo[9];
    pull_cell(P, A.fstar, x, y, f);  // pulled again from f*: cheaper than a stored copy
    for (int a = 0; a < 9; ++a) lo[a] = A.lf_in[a * pl + i];
    const float rho = A.rho[i], vx = A.vx[i], vy = A.vy[i];
    const float Fx = A.Fx[i], Fy = A.Fy[i], Fmx = A.Fmx[i], Fmy = A.Fmy[i], psi = A.psi[i];
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
    const float s = (rho - P.rho_v) * P.inv_drho;
    const float sfr = fminf(fmaxf(s, 0.f), 1.f);
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
    // ne_k = m_k(f) - meq_k(rho, v): m part -> lambda_f = M^T lambda_m
    float lf[9];
    {
        const float l1 = lne1, l2 = lne2, l4 = lne4, l6 = lne6, l7 = lne7, l8 = lne8;
        lf[0] = -4.f * l1 + 4.f * l2;
        lf[1] = -l1 - 2.f * l2 - 2.f * l4 + l7;
        lf[2] = -l1 - 2.f * l2 - 2.f * l6 - l7;
        lf[3] = -l1 - 2.f * l2 + 2.f * l4 + l7;
        lf[4] = -l1 - 2.f * l2 + 2.f * l6 - l7;
        lf[5] = 2.f * l1 + l2 + l4 + l6 + l8;
        lf[6] = 2.f * l1 + l2 - l4 + l6 - l8;
        lf[7] = 2.f * l1 + l2 - l4 - l6 + l8;
        lf[8] = 2.f * l1 + l2 + l4 - l6 - l8;
    }
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
    if (s > 0.f && s < 1.f) lrho += lsnu * (-snu * snu * P.dtau * P.inv_drho);
    // identity part of f* = f + ...
    for (int a = 0; a < 9; ++a) lf[a] += lo[a];
    // velocity v = (j + F/2) / rho with the thermal path's lambda_v added
    lvx += A.lvx[i] + lvx_c;
    lvy += A.lvy[i] + lvy_c;
    lrho += lr_c;
    const float irho = rcp_a(rho);
    const float ljx = lvx * irho, ljy = lvy * irho;
    lFx += 0.5f * ljx;
    lFy += 0.5f * ljy;
    lrho += -(lvx * vx + lvy * vy) * irho;
    for (int a = 0; a < 9; ++a) lf[a] += EXd[a] * ljx + EYd[a] * ljy;
    // forces: F = F_m + F_ads + F_b on fluid rows, 0 on wall rows
    if (!wall) {
        lFmx += lFx;
        lFmy += lFy;
        lrho += -P.g * lFy;  // F_b (Eq. 9)
        if (P.bc != BC_PERIODIC && y == 1) {  // F_ads (Eq. 22) on the first fluid row
            lpsi += 2.f * P.gw6 * psi * lFy;
            A.dGwx[x] += (double)(psi2 * (1.f / 6.f) * lFy);  // one cell per x on this row
        }
    } else {
        lFmx = lFmy = 0.f;  // no force is applied on wall rows
    }
    for (int a = 0; a < 9; ++a) A.lf[a * pl + i] = lf[a];
    A.lrho[i] += lrho;
    A.lpsi[i] = lpsi;
    A.lFmx[i] = lFmx;
    A.lFmy[i] = lFmy;
}

// F_m neighbour sums (Eq. 7) and psi (Eq. 21) transposed, the heat flux
// q(t) (in the window), rho = sum f; then the Zou-He fill transposed on the
// wall rows and the pull-streaming transposed. Writes lambda of f*^n and of
// theta^n.
__global__ void rev_psi(const StepParams P, AdjFields A, float lq) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    const bool wall = g.wall(y);
    const int pl = P.plane;
    const float psi = A.psi[i];
    float lpsi = A.lpsi[i];
    if (!wall) {  // own factor psi(x) of F_m(x) = -G psi(x) sum_a w_a psi(x + e_a) e_a
        float sx = 0.f, sy = 0.f;
        for (int a = 1; a < 9; ++a) {
            const float pn = A.psi[g.at(x, y, EXd[a], EYd[a])];
            sx += wdx(EXd[a], EYd[a]) * pn;
            sy += wdy(EXd[a], EYd[a]) * pn;
        }
        lpsi += -P.G * (sx * A.lFmx[i] + sy * A.lFmy[i]);
    }
    // neighbour factor: psi(y) appears in F_m(y - e_a); the eight lambda_F_m
    // pairs first (issued together), psi only where they are non-zero
    float lfx[9], lfy[9];
    int jj[9];
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        jj[a] = g.at(x, y, -EXd[a], -EYd[a]);
        lfx[a] = jj[a] < 0 ? 0.f : A.lFmx[jj[a]];
        lfy[a] = jj[a] < 0 ? 0.f : A.lFmy[jj[a]];
    }
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        if (lfx[a] == 0.f && lfy[a] == 0.f) continue;
        lpsi += -P.G * A.psi[jj[a]] * (wdx(EXd[a], EYd[a]) * lfx[a] + wdy(EXd[a], EYd[a]) * lfy[a]);
    }
    float lrho = A.lrho[i];
    float lth = A.lth[i];
    if (psi > 0.f) {
        const float rho = A.rho[i];
        const float T = P.Ts + A.theta[i];
        const Eos e = eos(rho, T, P);
        const float k = lpsi * rcp_a(P.G * psi);  // d psi = (dp - d rho / 3) / (G psi)
        lrho += k * (e.p_rho - 1.f / 3.f);
        lth += k * e.p_T;
    }
    // q(t) = (1/Lx) sum_x -cvchi rho(x,0) (-3 th0 + 4 th1 - th2) / 2 (Sec. 3.2)
    if (lq != 0.f && P.bc != BC_PERIODIC && y <= 2) {
        const float c = lq / (float)P.Lx * (-P.cvchi);
        const int i0 = x, i1 = P.pitch + x, i2 = 2 * P.pitch + x;
        const float rho0 = A.rho[i0];
        if (y == 0) {
            lrho += c * 0.5f * (-3.f * A.theta[i0] + 4.f * A.theta[i1] - A.theta[i2]);
            lth += c * rho0 * (-1.5f);
        } else if (y == 1) {
            lth += c * rho0 * 2.f;
        } else {
            lth += c * rho0 * (-0.5f);
        }
    }
    float lf[9];
    for (int a = 0; a < 9; ++a) lf[a] = A.lf[a * pl + i] + lrho;
    // Zou-He fill transposed: the filled populations pass their adjoint to
    // the known ones they were built from
    if (P.bc != BC_PERIODIC && y == 0) {
        lf[4] += lf[2];
        lf[7] += lf[5];
        lf[1] += -0.5f * lf[5] + 0.5f * lf[6];
        lf[3] += 0.5f * lf[5] - 0.5f * lf[6];
        lf[8] += lf[6];
        lf[2] = lf[5] = lf[6] = 0.f;
    }
    if (P.bc == BC_WALLS && y == P.Ly - 1) {
        lf[2] += lf[4];
        lf[5] += lf[7];
        lf[1] += 0.5f * lf[7] - 0.5f * lf[8];
        lf[3] += -0.5f * lf[7] + 0.5f * lf[8];
        lf[6] += lf[8];
        lf[4] = lf[7] = lf[8] = 0.f;
    }
    // pull-streaming transposed (f_a(y) = f*_a(y - e_a)) as a scatter:
    // lambda_f*_a(y - e_a) = lambda_f_a(y); a cell whose y + e_a lies beyond a
    // wall receives nothing and is set to 0 here
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const int t = g.at(x, y, -EXd[a], -EYd[a]);
        if (t >= 0) A.lf_out[a * pl + t] = lf[a];
        if (g.at(x, y, EXd[a], EYd[a]) < 0) A.lf_out[a * pl + i] = 0.f;
    }
    // the outflow top pulled populations 4, 7, 8 from its own row, whose
    // f* already has a consumer one row down: this second adjoint is kept in
    // the cell's own lf slot and added by outflow_push after this kernel
    if (P.bc == BC_TOP_OUTFLOW && y == P.Ly - 1) {
        A.lf[4 * pl + i] = lf[4];
        A.lf[7 * pl + i] = lf[7];
        A.lf[8 * pl + i] = lf[8];
    }
    A.lt_out[i] = lth;
}

// The outflow top's second consumer of f*_a(x - e_a, Ly - 1), a = 4, 7, 8.
__global__ void outflow_push(const StepParams P, AdjFields A) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.Lx) return;
    const int pl = P.plane, row = (P.Ly - 1) * P.pitch;
    const int a4[3] = {4, 7, 8};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = a4[k];
        int xs = x - EXd[a];
        if (xs < 0) xs += P.Lx;
        if (xs >= P.Lx) xs -= P.Lx;
        A.lf_out[a * pl + row + xs] += A.lf[a * pl + row + x];
    }
}

// Domains of at least this many cells recompute with the fused step (one
// launch instead of six; at 2048^2 the reverse step takes 0.83 ms instead of
// 0.96 ms); smaller ones with the field kernels (at 256^2 the six small
// launches take ~15 us, the fused step ~20 us).
constexpr size_t kFusedRecomputeCells = 512 * 512;

// Work-buffer layout: 39 field planes, then dJ/d theta_b [pitch doubles], the
// per-column dJ/dG_w parts [pitch doubles] and dJ/dG_w.
constexpr int kPlanes = 39;

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
    A.lf_in = A.lt_in = nullptr;
    A.lf_out = A.lt_out = nullptr;
    A.rho = next(1);
    A.psi = next(1);
    A.jx = next(1);
    A.jy = next(1);
    A.Fmx = next(1);
    A.Fmy = next(1);
    A.Fx = next(1);
    A.Fy = next(1);
    A.vx = next(1);
    A.vy = next(1);
    A.drx = next(1);
    A.dry = next(1);
    A.divv = next(1);
    A.ax = next(1);
    A.ay = next(1);
    A.cA = next(1);
    A.cB = next(1);
    A.u2 = next(1);
    A.u3 = next(1);
    A.u4 = next(1);
    A.lf = next(9);
    A.lrho = next(1);
    A.lpsi = next(1);
    A.lFmx = next(1);
    A.lFmy = next(1);
    A.lvx = next(1);
    A.lvy = next(1);
    A.lth = next(1);
    A.ldrx = next(1);
    A.ldry = next(1);
    A.ldivv = next(1);
    A.dTb = (double*)(w + kPlanes * pl);
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
    return sizeof(float) * (size_t)kPlanes * (size_t)P.plane + sizeof(double) * (2 * (size_t)P.pitch + 2);
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

// One reverse step: state (fstar, theta) of level n, lambda of level n+1 in
// (lf_in, lt_in), lambda of level n out; lq = dJ/dq(t_n). L is a dual-strip
// launch shape matching P (nout, nstrips, seg_h) for the recompute.
cudaError_t adjoint_reverse_step(const StepParams& P, const Launch& L, void* work, const float* fstar,
                                 const float* theta, const float* lf_in, const float* lt_in, float* lf_out,
                                 float* lt_out, float lq, cudaStream_t st) {
    AdjFields A = fields_at(P, work);
    A.fstar = fstar;
    A.theta = theta;
    A.lf_in = lf_in;
    A.lt_in = lt_in;
    A.lf_out = lf_out;
    A.lt_out = lt_out;
    // 32 x 8 tiles: the vertical neighbours of a warp's cells are read by the
    // warps above and below it in the same block, so they stay in L1
    const dim3 blk(32, 8), grid((P.Lx + 31) / 32, (P.Ly + 7) / 8);
    // the step's intermediates from (f*^n, theta^n): written by the fused step
    // on large domains, by the field kernels above on small ones
    StepParams Q = P;
    Q.f_in = fstar;
    Q.th_in = theta;
    Q.f_out = nullptr;
    Q.th_out = nullptr;
    const RecomputeOut R{A.rho, A.psi, A.jx, A.jy, A.Fmx, A.Fmy, A.Fx, A.Fy, A.vx, A.vy,
                         A.drx, A.dry, A.divv, A.ax, A.ay, A.cA, A.cB, A.u2, A.u3, A.u4};
    if ((size_t)P.Lx * P.Ly >= kFusedRecomputeCells) {
        cudaError_t e = dual_recompute(Q, R, L, st);
        if (e != cudaSuccess) return e;
    } else {
        fwd_pull<<<grid, blk, 0, st>>>(P, A);
        fwd_force<<<grid, blk, 0, st>>>(P, A);
        fwd_coef<<<grid, blk, 0, st>>>(P, A);
        fwd_stage<<<grid, blk, 0, st>>>(P, A, theta, A.u2, 0.5f);
        fwd_stage<<<grid, blk, 0, st>>>(P, A, A.u2, A.u3, 0.5f);
        fwd_stage<<<grid, blk, 0, st>>>(P, A, A.u3, A.u4, 1.0f);
    }
    // the four RK stages transposed: one column-marching launch, segments
    // sized so that the blocks fill the GPU once
    {
        static int occ = 0, nsm = 0;
        cudaError_t e = cudaSuccess;
        if (!occ) {
            int dev = 0;
            e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) e = cudaFuncSetAttribute(rev_thermal_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)rt_smem_bytes());
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rev_thermal_fused, RT_BD, rt_smem_bytes());
            if (e != cudaSuccess) return e;
            occ = occ < 1 ? 1 : occ;
        }
        const int nstrips = (P.Lx + RT_BD - 2 * RT_HALO - 1) / (RT_BD - 2 * RT_HALO);
        const int nseg = std::max(1, nsm * occ / nstrips);
        const int seg_h = std::max(16, (P.Ly + nseg - 1) / nseg);
        const int nb = nstrips * ((P.Ly + seg_h - 1) / seg_h);
        rev_thermal_fused<<<nb, RT_BD, rt_smem_bytes(), st>>>(P, A, seg_h);
    }
    rev_collide<<<grid, blk, 0, st>>>(P, A);
    rev_psi<<<grid, blk, 0, st>>>(P, A, lq);
    if (P.bc == BC_TOP_OUTFLOW) outflow_push<<<(P.Lx + 127) / 128, 128, 0, st>>>(P, A);
    return cudaGetLastError();
}

}  // namespace lbgpu
