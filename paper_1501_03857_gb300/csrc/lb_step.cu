// The fused time step: pull-stream, Zou-He walls, pseudopotential force,
// MRT collision with the improved forcing term, RK4 temperature update and
// the bottom-wall heat-flux reduction, in one kernel.
//
// Design (GB300): a block owns a strip of (blockDim - 10) output columns and
// a segment of rows, and marches up the segment one row per iteration. Each
// thread owns one column (5 halo columns on each side are recomputed, not
// exchanged). The stencil quantities of the last few rows (psi, rho, v and
// the three RK stage inputs) live in shared-memory ring buffers, so every
// population and temperature value is read from HBM once and written once
// per step. The work of one iteration is a pipeline over consecutive rows:
//
//   P  row L    : pull f (loads issued one iteration ahead), wall fill,
//                 rho, psi(rho, T^t)                       (Eqs. 3, 6, 21)
//   B  row L-1  : F_m, F_ads, F_b, v, MRT collision, store f*   (Eqs. 2-9, 22)
//   C  row L-2  : grad rho, div v, RK stage 1 of Eq. 18        (Eqs. 18-20)
//   D  row L-3  : RK stage 2
//   E  row L-4  : RK stage 3
//   F  row L-5  : RK stage 4, store theta^{t+1}
//
// A row's value in stage k needs only rows +-1 of stage k-1, so the rows a
// segment computes shrink by one per stage from [ys-5, ye+5) to [ys, ye).
#include "lb_internal.h"

namespace lbgpu {

namespace {

// Isotropic central differences (Lee and Lin; Sec. 2 after Eq. 20) on the
// 3x3 neighbourhood of column s in rows m (y-1), c (y), p (y+1).
struct Stencil {
    float dx, dy, lap, c;
};

__device__ __forceinline__ Stencil stencil(const float* __restrict__ m, const float* __restrict__ c,
                                           const float* __restrict__ p) {
    const float W = c[-1], C = c[0], E = c[1];
    const float SW = m[-1], S = m[0], SE = m[1];
    const float NW = p[-1], N = p[0], NE = p[1];
    Stencil o;
    o.dx = (E - W) * (1.f / 3.f) + ((NE - SW) + (SE - NW)) * (1.f / 12.f);
    o.dy = (N - S) * (1.f / 3.f) + ((NE - SW) + (NW - SE)) * (1.f / 12.f);
    o.lap = (4.f * (E + W + N + S) + (NE + NW + SE + SW) - 20.f * C) * (1.f / 6.f);
    o.c = C;
    return o;
}

// Per-cell coefficients of K(T) (Eq. 18) with rho and v frozen at level t:
// K = ax dT/dx + ay dT/dy + chi lap T - T (cA - cB phi'(T)), where
// ax = -v_x + chi d_x rho / rho (from div(lambda grad T)/(rho c_v) with
// lambda = c_v chi rho) and cA - cB phi' = (dp/dT)_rho div v / (rho c_v).
struct Coef {
    float ax, ay, cA, cB;
};

__device__ __forceinline__ float rhs_K(const Stencil& u, const Coef& k, const StepParams& P) {
    const float T = P.Ts + u.c;
    const float sT = sqrtf(T);
    const float dphi = -P.k1 * (P.k0 - P.k1 * sT) / sT;  // phi'(T), Eq. 21
    return k.ax * u.dx + k.ay * u.dy + P.chi * u.lap - T * (k.cA - k.cB * dphi);
}

// MRT collision, Eq. 2, with the forcing moments of Eq. 8, written in the
// exactly equivalent additive form f* = f + M^-1 dm with
// dm = -Lambda (m - m^eq) + (I - Lambda/2) S. dm is small (non-equilibrium
// moments and forces), so FP32 rounding stays at ~1 ulp of f per step and
// mass is conserved to rounding (dm_rho = 0 exactly). The non-equilibrium
// moments use rho v = j + F/2 (Eq. 6) in place of the rounded product.
__device__ __forceinline__ void collide_store(const float (&f)[9], float rho, float vx, float vy,
                                              float Fx, float Fy, float Fmx, float Fmy, float psi,
                                              const StepParams& P, float* __restrict__ out, int idx) {
    const float sa = (f[1] + f[3]) + (f[2] + f[4]);
    const float sd = (f[5] + f[7]) + (f[6] + f[8]);
    const float dxd = (f[5] - f[7]) + (f[8] - f[6]);  // sum of e_x f over diagonals
    const float dyd = (f[5] - f[7]) + (f[6] - f[8]);  // sum of e_y f over diagonals
    const float v2 = vx * vx + vy * vy;
    const float rv2 = rho * v2;
    // m - m^eq (Eq. 5) for e, zeta, qx, qy, pxx, pxy
    const float ne1 = (sa + 4.f * sd - 2.f * f[0]) - 3.f * rv2;
    const float ne2 = 3.f * (f[0] - sa) + 3.f * rv2;
    const float ne4 = 2.f * dxd - (f[1] - f[3]) + 0.5f * Fx;
    const float ne6 = 2.f * dyd - (f[2] - f[4]) + 0.5f * Fy;
    const float ne7 = ((f[1] + f[3]) - (f[2] + f[4])) - rho * (vx * vx - vy * vy);
    const float ne8 = ((f[5] + f[7]) - (f[6] + f[8])) - rho * vx * vy;
    // S, Eq. 8
    const float vF = vx * Fx + vy * Fy;
    const float psi2 = psi * psi;
    const float ratio = psi2 > 0.f ? (Fmx * Fmx + Fmy * Fmy) / psi2 : 0.f;
    const float S1 = 6.f * vF + P.sig_e * ratio;
    const float S2 = -6.f * vF - P.sig_z * ratio;
    const float S7 = 2.f * (vx * Fx - vy * Fy);
    const float S8 = vx * Fy + vy * Fx;
    // tau_nu(rho): linear between the coexistence densities, clamped
    const float sfr = fminf(fmaxf((rho - P.rho_v) * P.inv_drho, 0.f), 1.f);
    const float snu = 1.f / (P.tau_v + P.dtau * sfr);
    // dm = -Lambda (m - m^eq) + (I - Lambda/2) S; with s_j = 1 and
    // rho v = j + F/2 the momentum rows give dm_j = F.
    const float dm1 = -P.s_e * ne1 + (1.f - 0.5f * P.s_e) * S1;
    const float dm2 = -P.s_z * ne2 + (1.f - 0.5f * P.s_z) * S2;
    const float dm4 = -P.s_q * ne4 - (1.f - 0.5f * P.s_q) * Fx;
    const float dm6 = -P.s_q * ne6 - (1.f - 0.5f * P.s_q) * Fy;
    const float dm7 = -snu * ne7 + (1.f - 0.5f * snu) * S7;
    const float dm8 = -snu * ne8 + (1.f - 0.5f * snu) * S8;
    // M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const float n1 = dm1 * (1.f / 36.f), n2 = dm2 * (1.f / 36.f);
    const float n3 = Fx * (1.f / 6.f), n4 = dm4 * (1.f / 12.f);
    const float n5 = Fy * (1.f / 6.f), n6 = dm6 * (1.f / 12.f);
    const float n7 = dm7 * 0.25f, n8 = dm8 * 0.25f;
    const float ax_ = -n1 - 2.f * n2;
    const float dg = 2.f * n1 + n2;
    const float cx = n3 - 2.f * n4, cy = n5 - 2.f * n6;
    const float dxx = n3 + n4, dyy = n5 + n6;
    const int pl = P.plane;
    out[idx] = f[0] + (4.f * (n2 - n1));
    out[1 * pl + idx] = f[1] + (ax_ + cx + n7);
    out[2 * pl + idx] = f[2] + (ax_ + cy - n7);
    out[3 * pl + idx] = f[3] + (ax_ - cx + n7);
    out[4 * pl + idx] = f[4] + (ax_ - cy - n7);
    out[5 * pl + idx] = f[5] + (dg + dxx + dyy + n8);
    out[6 * pl + idx] = f[6] + (dg - dxx + dyy - n8);
    out[7 * pl + idx] = f[7] + (dg - dxx - dyy + n8);
    out[8 * pl + idx] = f[8] + (dg + dxx - dyy - n8);
}

}  // namespace

__global__ void __launch_bounds__(512, 1) lb_fused_step(const StepParams P) {
    extern __shared__ float smem[];
    __shared__ double red[32];
    const int BD = blockDim.x, W = BD + 2;
    float* const sPSI = smem;
    float* const sRHO = sPSI + RING * W;
    float* const sVX = sRHO + RING * W;
    float* const sVY = sVX + RING * W;
    float* const sU2 = sVY + RING * W;
    float* const sU3 = sU2 + RING * W;
    float* const sU4 = sU3 + RING * W;
    float* const sTH = sU4 + RING * W;
    for (int i = threadIdx.x; i < SM_ROWS * W; i += BD) smem[i] = 0.f;

    const int Lx = P.Lx, Ly = P.Ly;
    const int strip = blockIdx.x % P.nstrips;
    const int seg = blockIdx.x / P.nstrips;
    const int x0 = strip * P.nout;
    const int nvalid = min(P.nout, Lx - x0);
    const int lc = threadIdx.x;
    const int s = lc + 1;
    const int x = wrap(x0 - HALO + lc, Lx);
    const int xm = x == 0 ? Lx - 1 : x - 1;
    const int xp = x == Lx - 1 ? 0 : x + 1;
    const bool outc = lc >= HALO && lc < HALO + nvalid;
    const bool periodic = P.bc == BC_PERIODIC;
    const int ys = seg * P.seg_h;
    const int ye = min(ys + P.seg_h, Ly);
    // pipeline row range of each stage
    auto lo = [&](int d) { return periodic ? ys - d : max(ys - d, 0); };
    auto hi = [&](int d) { return periodic ? ye + d : min(ye + d, Ly); };
    const int loP = lo(5), hiP = hi(5), loB = lo(4), hiB = hi(4), loC = lo(3), hiC = hi(3);
    const int loD = lo(2), hiD = hi(2), loE = lo(1), hiE = hi(1);
    const bool thermal = !P.isothermal;
    bool eos_bad = false, nonfinite = false;

    float fc[9], tc = 0.f;
    if (loP < hiP) load_row(P, wrap(loP, Ly), x, xm, xp, fc, tc);

    float fP[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float rhoP = 1.f, jxP = 0.f, jyP = 0.f, psiP = 0.f;
    Coef k1{0.f, 0.f, 0.f, 0.f}, k2 = k1, k3 = k1;
    float acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
    __syncthreads();

    for (int L = loP; L <= ye + 4; ++L) {
        // ---- prefetch the pulled populations of row L+1
        float fn[9], tn = 0.f;
        const bool nextP = (L + 1 < hiP);
        if (nextP) load_row(P, wrap(L + 1, Ly), x, xm, xp, fn, tn);

        // ---- P: wall fill, rho, psi of row L
        float fN[9], rhoN = 1.f, jxN = 0.f, jyN = 0.f, psiN = 0.f;
        if (L < hiP) {
            const int y = wrap(L, Ly);
#pragma unroll
            for (int a = 0; a < 9; ++a) fN[a] = fc[a];
            wall_fill(P, y, fN);
            rhoN = ((fN[0] + fN[1]) + (fN[2] + fN[3])) + ((fN[4] + fN[5]) + (fN[6] + fN[7])) + fN[8];
            jxN = (fN[1] - fN[3]) + (fN[5] - fN[6]) + (fN[8] - fN[7]);
            jyN = (fN[2] - fN[4]) + (fN[5] + fN[6]) - (fN[7] + fN[8]);
            psiN = eos_psi(rhoN, P.Ts + tc, P, eos_bad);
            sPSI[(L & 3) * W + s] = psiN;
            sRHO[(L & 3) * W + s] = rhoN;
            sTH[(L & 7) * W + s] = tc;
        }
        __syncthreads();

        // ---- bottom-wall heat flux of level t (Sec. 3.2), one sample per step
        if (!periodic && ys == 0 && L == 2) {
            double q = 0.0;
            if (outc) {
                const double r0 = sRHO[0 * W + s];
                const double t0 = sTH[0 * W + s], t1 = sTH[1 * W + s], t2 = sTH[2 * W + s];
                q = -(double)P.cvchi * r0 * (-3.0 * t0 + 4.0 * t1 - t2) * 0.5;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
            if ((lc & 31) == 0) red[lc >> 5] = q;
            __syncthreads();
            if (lc == 0) {
                double sum = 0.0;
                for (int w = 0; w < (BD >> 5); ++w) sum += red[w];
                Acc* A = P.acc;
                atomicAdd(&A->q_partial, sum);
                __threadfence();
                const unsigned t = atomicAdd(&A->count, 1u);
                if (t == (unsigned)P.nstrips - 1u) {
                    __threadfence();
                    const double tot = __longlong_as_double(
                        (long long)atomicExch((unsigned long long*)&A->q_partial, 0ull));
                    const double qt = tot / (double)Lx;
                    A->q_last = qt;
                    A->q_sum += qt;
                    A->q_sum2 += qt * qt;
                    A->q_n += 1.0;
                    atomicExch(&A->count, 0u);
                }
            }
        }

        // ---- B: forces, velocity, collision of row L-1
        {
            const int r = L - 1;
            if (r >= loB && r < hiB) {
                const int y = wrap(r, Ly);
                const bool wall = !periodic && (y == 0 || y == Ly - 1);
                float Fmx = 0.f, Fmy = 0.f;
                if (!wall || P.ghost) {
                    const float* pc = sPSI + (r & 3) * W + s;
                    const float* pn = (wall && y == Ly - 1) ? pc : sPSI + ((r + 1) & 3) * W + s;
                    const float* ps = (wall && y == 0) ? pc : sPSI + ((r - 1) & 3) * W + s;
                    float sx, sy;
                    psi_sum(ps, pc, pn, sx, sy);
                    Fmx = -P.G * psiP * sx;
                    Fmy = -P.G * psiP * sy;
                }
                float Fx = Fmx, Fy = Fmy;
                if (!wall) {
                    if (!periodic && y == 1) Fy += P.gw6 * psiP * psiP;  // Eq. 22
                    Fy -= P.g * (rhoP - P.rho_ave);                       // Eq. 9
                }
                const float inv_rho = 1.f / rhoP;
                const float vx = (jxP + 0.5f * Fx) * inv_rho;  // Eq. 6
                const float vy = (jyP + 0.5f * Fy) * inv_rho;
                sVX[(r & 3) * W + s] = vx;
                sVY[(r & 3) * W + s] = vy;
                if (outc && r >= ys && r < ye) {
                    if (!finite_f(rhoP)) nonfinite = true;
                    collide_store(fP, rhoP, vx, vy, Fx, Fy, Fmx, Fmy, psiP, P, P.f_out,
                                  y * P.pitch + x);
                }
            }
        }
        __syncthreads();

        // Stage C makes the coefficients of row L-2; stages D, E, F of this
        // iteration work on rows whose coefficients C made 1, 2 and 3
        // iterations ago (carried in k1/acc1, k2/acc2, k3/acc3).
        Coef kC{0.f, 0.f, 0.f, 0.f};
        float accC = 0.f;
        if (thermal) {
            // ---- C: frozen-flow coefficients and RK stage 1 of row L-2
            {
                const int r = L - 2;
                if (r >= loC && r < hiC) {
                    const int y = wrap(r, Ly);
                    const float thr = sTH[(r & 7) * W + s];
                    float u2 = thr;
                    if (periodic || (y != 0 && y != Ly - 1)) {
                        const int sm = ((r - 1) & 3) * W + s, sc = (r & 3) * W + s,
                                  sp = ((r + 1) & 3) * W + s;
                        const Stencil gr = stencil(sRHO + sm, sRHO + sc, sRHO + sp);
                        const Stencil gvx = stencil(sVX + sm, sVX + sc, sVX + sp);
                        const Stencil gvy = stencil(sVY + sm, sVY + sc, sVY + sp);
                        const float rho = gr.c;
                        const float inv_rho = 1.f / rho;
                        const float divv = gvx.dx + gvy.dy;
                        const float br = P.b * rho;
                        kC.ax = -gvx.c + P.chi * gr.dx * inv_rho;
                        kC.ay = -gvy.c + P.chi * gr.dy * inv_rho;
                        kC.cA = divv * P.R * P.inv_cv / (1.f - br);
                        kC.cB = divv * P.a * rho * P.inv_cv / (1.f + 2.f * br - br * br);
                        const int tm = ((r - 1) & 7) * W + s, tcn = (r & 7) * W + s,
                                  tp = ((r + 1) & 7) * W + s;
                        accC = rhs_K(stencil(sTH + tm, sTH + tcn, sTH + tp), kC, P);
                        u2 = thr + 0.5f * accC;
                    }
                    sU2[(r & 3) * W + s] = u2;
                }
            }
            __syncthreads();
            // ---- D: RK stage 2 of row L-3
            {
                const int r = L - 3;
                if (r >= loD && r < hiD) {
                    const int y = wrap(r, Ly);
                    const float thr = sTH[(r & 7) * W + s];
                    float u3 = thr;
                    if (periodic || (y != 0 && y != Ly - 1)) {
                        const int sm = ((r - 1) & 3) * W + s, sc = (r & 3) * W + s,
                                  sp = ((r + 1) & 3) * W + s;
                        const float h2 = rhs_K(stencil(sU2 + sm, sU2 + sc, sU2 + sp), k1, P);
                        u3 = thr + 0.5f * h2;
                        acc1 += 2.f * h2;
                    }
                    sU3[(r & 3) * W + s] = u3;
                }
            }
            __syncthreads();
            // ---- E: RK stage 3 of row L-4
            {
                const int r = L - 4;
                if (r >= loE && r < hiE) {
                    const int y = wrap(r, Ly);
                    const float thr = sTH[(r & 7) * W + s];
                    float u4 = thr;
                    if (periodic || (y != 0 && y != Ly - 1)) {
                        const int sm = ((r - 1) & 3) * W + s, sc = (r & 3) * W + s,
                                  sp = ((r + 1) & 3) * W + s;
                        const float h3 = rhs_K(stencil(sU3 + sm, sU3 + sc, sU3 + sp), k2, P);
                        u4 = thr + h3;
                        acc2 += 2.f * h3;
                    }
                    sU4[(r & 3) * W + s] = u4;
                }
            }
            __syncthreads();
        }
        // ---- F: RK stage 4 and theta^{t+1} of row L-5
        {
            const int r = L - 5;
            if (r >= ys && r < ye && outc) {
                const int y = wrap(r, Ly);
                const float thr = sTH[(r & 7) * W + s];
                float tnew = thr;
                if (thermal) {
                    if (!periodic && y == 0) {
                        tnew = __ldg(P.thb + x);
                    } else if (!periodic && y == Ly - 1) {
                        tnew = 0.f;
                    } else {
                        const int sm = ((r - 1) & 3) * W + s, sc = (r & 3) * W + s,
                                  sp = ((r + 1) & 3) * W + s;
                        const float h4 = rhs_K(stencil(sU4 + sm, sU4 + sc, sU4 + sp), k3, P);
                        tnew = thr + (acc3 + h4) * (1.f / 6.f);
                    }
                }
                if (!finite_f(tnew)) nonfinite = true;
                P.th_out[y * P.pitch + x] = tnew;
            }
        }
        k3 = k2;
        acc3 = acc2;
        k2 = k1;
        acc2 = acc1;
        k1 = kC;
        acc1 = accC;
        // rotate per-thread carries
#pragma unroll
        for (int a = 0; a < 9; ++a) fP[a] = fN[a];
        rhoP = rhoN;
        jxP = jxN;
        jyP = jyN;
        psiP = psiN;
#pragma unroll
        for (int a = 0; a < 9; ++a) fc[a] = fn[a];
        tc = tn;
    }
    if (eos_bad) atomicOr(&P.acc->err, ERR_EOS);
    if (nonfinite) atomicOr(&P.acc->err, ERR_NONFINITE);
}

size_t step_smem_bytes(int block_x) { return sizeof(float) * (size_t)SM_ROWS * (size_t)(block_x + 2); }

cudaError_t step_prepare(int block_x) {
    return cudaFuncSetAttribute(lb_fused_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step_smem_bytes(block_x));
}

int step_occupancy(int block_x, int* blocks_per_sm) {
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, lb_fused_step, block_x,
                                                              step_smem_bytes(block_x));
}

cudaError_t launch_step(const StepParams& P, const Launch& L, cudaStream_t st) {
    if (L.kernel == KERNEL_PAIRS) return pairs_launch(P, L, st);
    if (L.kernel == KERNEL_DUAL) return dual_launch(P, L, true, st);
    if (L.kernel == KERNEL_DUAL_SCALAR) return dual_launch(P, L, false, st);
    lb_fused_step<<<L.nstrips * L.nseg, L.block_x, step_smem_bytes(L.block_x), st>>>(P);
    return cudaGetLastError();
}

}  // namespace lbgpu
