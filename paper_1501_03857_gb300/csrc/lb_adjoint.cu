// Discrete adjoint of one time step (reverse mode), for gradients of the
// time-averaged bottom-wall heat flux J = (1/S) sum_n q(t_n) (Sec. 3.2) with
// respect to the wall temperature profile T_b(x) and the wettability G_w of
// Eq. 22.
//
// Forward intermediates of step n are recomputed from the stored state
// (f*^n, theta^n): on large domains by the fused step itself in its
// recompute mode (lb_step3.cu, RecomputeOut), on small ones by field kernels
// (one thread per cell) that follow its formulas. The reverse passes (field
// kernels) then transpose each part of the step in the opposite order:
//
//   RK4 of Eq. 18 (stage 4 .. 1)   -> lambda_theta, lambda of the per-cell
//                                     coefficients (ax, ay, cA, cB)
//   coefficients                   -> lambda_rho, lambda_v (grad rho, div v)
//   MRT collision (Eqs. 2, 5, 8), v (Eq. 6), forces (Eqs. 7, 9, 22)
//                                  -> lambda_f, lambda_rho, lambda_psi, lambda_F_m
//   F_m neighbour sums (Eq. 7), psi (Eq. 21), q_w, rho = sum f
//                                  -> lambda_f, lambda_theta
//   Zou-He fill, pull-streaming (Eq. 3)
//                                  -> lambda_f*^n
//
// A stencil applied forward as out(x) = sum_d c_d in(x + d) is transposed as
// a gather lambda_in(y) += sum_d c_d lambda_out(y - d). Fields are pitched
// [Ly][pitch] FP32; gradients are accumulated in FP64. Supported: walls or
// periodic in y, no ghost layer (the host checks).
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
    float *lax, *lay, *lcA, *lcB, *mu, *mu_next, *ldrx, *ldry, *ldivv;
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
__device__ __forceinline__ void rev_coef_cell(const StepParams& P, const AdjFields& A, int i, bool wall) {
    if (wall) {
        A.ldrx[i] = A.ldry[i] = A.ldivv[i] = 0.f;
        A.lrho[i] = A.lvx[i] = A.lvy[i] = 0.f;
        return;
    }
    const float rho = A.rho[i], irho = rcp_a(rho);
    const float lax = A.lax[i], lay = A.lay[i], lcA = A.lcA[i], lcB = A.lcB[i];
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

// Transpose of one RK stage h = mask K(u): from mu (= mask lambda_h) compute
// lambda_u (transposed stencils + the diagonal source term), accumulate the
// coefficient adjoints and lambda_theta (u = theta + ...), and form the next
// stage's mu = mask (a lambda-bar + b lambda_u). The first (stage 4) starts
// the sweep: its mu is lambda-bar / 6 with lambda-bar the incoming
// lambda_theta on fluid rows, the accumulators start from lambda-bar
// (identity part of theta' = theta + ...) and 0, and the incoming lambda of
// the new bottom wall row (its Dirichlet value) goes to dJ/d theta_b.
__global__ void rev_stage(const StepParams P, AdjFields A, const float* u, float a_bar, float b_u, int first,
                          int last) {
    int x, y, i;
    if (!cell(P, x, y, i)) return;
    const Grid g = grid_of(P);
    const bool wall = g.wall(y);
    auto mu_at = [&](int j, int yj) {
        return first ? (g.wall(yj) ? 0.f : A.lt_in[j] * (1.f / 6.f)) : A.mu[j];
    };
    // the nine neighbours' mu first (issued together), then their
    // coefficients only where mu is non-zero: lambda is zero away from the
    // heated wall early in a reverse sweep, and those cells cost no traffic
    float mj[9];
    int jj[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        // source cell s = y - d with d = e_a contributes c_d(s) mu(s)
        jj[a] = g.at(x, y, -EXd[a], -EYd[a]);
        mj[a] = jj[a] < 0 ? 0.f : mu_at(jj[a], y - EYd[a]);
    }
    float lu = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        if (mj[a] == 0.f) continue;
        const int j = jj[a], dx = EXd[a], dy = EYd[a];
        lu += (A.ax[j] * wdx(dx, dy) + A.ay[j] * wdy(dx, dy) + P.chi * wlap(dx, dy)) * mj[a];
    }
    const float m = mj[0];  // own cell (e_0 = 0)
    float lax = 0.f, lay = 0.f, lcA = 0.f, lcB = 0.f;
    if (!wall && m != 0.f) {
        const float T = P.Ts + u[i];
        const float rs = rsqrt_a(T);
        const float dphi = P.k1k1 - P.k0k1 * rs;
        const float d2phi = 0.5f * P.k0k1 * (rs * rs * rs);
        lu += (-(A.cA[i] - A.cB[i] * dphi) + T * A.cB[i] * d2phi) * m;
        float dx = 0.f, dy = 0.f;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const float un = u[g.at(x, y, EXd[a], EYd[a])];
            dx += wdx(EXd[a], EYd[a]) * un;
            dy += wdy(EXd[a], EYd[a]) * un;
        }
        lax = dx * m;
        lay = dy * m;
        lcA = -T * m;
        lcB = T * dphi * m;
    }
    if (first) {
        const float lin = A.lt_in[i];
        if (P.bc != BC_PERIODIC && y == 0) A.dTb[x] += (double)lin;
        A.lax[i] = lax;
        A.lay[i] = lay;
        A.lcA[i] = lcA;
        A.lcB[i] = lcB;
        A.lth[i] = (wall ? 0.f : lin) + lu;
    } else {
        if (lax != 0.f || lay != 0.f || lcA != 0.f || lcB != 0.f) {
            A.lax[i] += lax;
            A.lay[i] += lay;
            A.lcA[i] += lcA;
            A.lcB[i] += lcB;
        }
        A.lth[i] += lu;
    }
    if (!last) {
        const float lin = A.lt_in[i];
        const float lbar = wall ? 0.f : lin;
        A.mu_next[i] = wall ? 0.f : (a_bar * lbar + b_u * lu);
    } else {
        rev_coef_cell(P, A, i, wall);
    }
}

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
    A.lt_out[i] = lth;
}

// Domains of at least this many cells recompute with the fused step (one
// launch instead of six; at 2048^2 the reverse step takes 0.83 ms instead of
// 0.96 ms); smaller ones with the field kernels (at 256^2 the six small
// launches take ~15 us, the fused step ~20 us).
constexpr size_t kFusedRecomputeCells = 512 * 512;

// Work-buffer layout: 45 field planes, then dJ/d theta_b [pitch doubles], the
// per-column dJ/dG_w parts [pitch doubles] and dJ/dG_w.
constexpr int kPlanes = 45;

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
    A.lax = next(1);
    A.lay = next(1);
    A.lcA = next(1);
    A.lcB = next(1);
    A.mu = next(1);
    A.mu_next = next(1);
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
    const float* us[4] = {A.u4, A.u3, A.u2, theta};
    const float abar[4] = {1.f / 3.f, 1.f / 3.f, 1.f / 6.f, 0.f};
    const float bu[4] = {1.f, 0.5f, 0.5f, 0.f};
    for (int k = 0; k < 4; ++k) {
        rev_stage<<<grid, blk, 0, st>>>(P, A, us[k], abar[k], bu[k], k == 0, k == 3);
        float* t = A.mu;
        A.mu = A.mu_next;
        A.mu_next = t;
    }
    rev_collide<<<grid, blk, 0, st>>>(P, A);
    rev_psi<<<grid, blk, 0, st>>>(P, A, lq);
    return cudaGetLastError();
}

}  // namespace lbgpu
