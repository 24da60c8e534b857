// The fused time step, two rows per iteration with paired FP32 arithmetic.
//
// Same pipeline as the row-wise kernel (lb_step.cu): a block owns a strip of
// (BD - 10) output columns and a segment of rows and marches up it; every
// population and temperature value is read from HBM once and written once.
// Here each iteration advances a PAIR of rows, and the two cells a thread
// holds for a column (rows 2q and 2q+1) are packed into one float2. The
// cell-local arithmetic (EOS, forces, MRT collision, RK coefficients and
// stage updates) then runs on Blackwell's paired FP32 instructions
// (__ffma2_rn / __fadd2_rn / __fmul2_rn: two FP32 operations per issue
// slot), and barriers, loop and ring-index overhead are paid once per two
// rows. Reciprocals and square roots use the MUFU approximations
// (__fdividef, rsqrtf; <= 2 ulp).
//
// Stages of iteration q (pair p = rows 2p, 2p+1):
//   P  pair q   : wall fill, rho, psi(rho, T^t)                 (Eqs. 3, 6, 21)
//   B  pair q-1 : F_m, F_ads, F_b, v, MRT collision, store f*   (Eqs. 2-9, 22)
//   C  pair q-2 : grad rho, div v, RK stage 1                   (Eqs. 18-20)
//   D  pair q-3 : RK stage 2
//   E  pair q-4 : RK stage 3
//   F  pair q-5 : RK stage 4, store theta^{t+1}
// The pulled populations of pair q+1 are loaded during stages C-F.
#include "lb_internal.h"

namespace lbgpu {

namespace {

typedef float2 v2;

__device__ __forceinline__ v2 bc(float s) { return make_float2(s, s); }
__device__ __forceinline__ v2 operator+(v2 a, v2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ v2 operator-(v2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ v2 operator-(v2 a, v2 b) { return __fadd2_rn(a, -b); }
__device__ __forceinline__ v2 operator*(v2 a, v2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ v2 operator*(float s, v2 b) { return __fmul2_rn(bc(s), b); }
__device__ __forceinline__ v2 fma2(v2 a, v2 b, v2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ v2 rcp2(v2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
__device__ __forceinline__ v2 rsqrt2(v2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ v2 sel(bool px, bool py, v2 a, v2 b) {  // per component: p ? a : b
    return make_float2(px ? a.x : b.x, py ? a.y : b.y);
}

// Pulled populations and theta of the row pair starting at pipeline row R0
// (rows outside a wall-bounded domain read as 0 and are never used).
__device__ __forceinline__ void load_pair(const StepParams& P, int R0, int x, int xm, int xp, v2 (&f)[9], v2& th) {
    float a[9], b[9], ta = 0.f, tb = 0.f;
    const bool per = P.bc == BC_PERIODIC;
    if (per || (R0 >= 0 && R0 < P.Ly)) {
        load_row(P, wrap(R0, P.Ly), x, xm, xp, a, ta);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) a[k] = 0.f;
    }
    if (per || (R0 + 1 >= 0 && R0 + 1 < P.Ly)) {
        load_row(P, wrap(R0 + 1, P.Ly), x, xm, xp, b, tb);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) b[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) f[k] = make_float2(a[k], b[k]);
    th = make_float2(ta, tb);
}

// psi of Sec. 2 with the PR EOS of Eq. 21, for a pair of cells.
__device__ __forceinline__ v2 eos_psi2(v2 rho, v2 T, const StepParams& P, bool& bad) {
    const v2 sT = T * rsqrt2(T);
    v2 ph = fma2(bc(-P.k1), sT, bc(P.k0));
    ph = ph * ph;
    const v2 br = P.b * rho;
    const v2 i1 = rcp2(bc(1.f) - br);
    const v2 i2 = rcp2(fma2(br, bc(2.f) - br, bc(1.f)));  // 1 + 2 b rho - b^2 rho^2
    const v2 p = (P.R * rho) * T * i1 - (P.a * ph) * (rho * rho) * i2;
    const v2 arg = P.two_over_G * fma2(rho, bc(-1.f / 3.f), p);
    bad |= (arg.x < 0.f) | (arg.y < 0.f);
    return make_float2(arg.x > 0.f ? arg.x * rsqrtf(arg.x) : 0.f, arg.y > 0.f ? arg.y * rsqrtf(arg.y) : 0.f);
}

// Isotropic central differences (Lee and Lin; Sec. 2 after Eq. 20) for the
// pair at column s of ring slot `cur`, with the row below the pair in slot
// `prv` (its .y) and the row above in slot `nxt` (its .x).
struct St2 {
    v2 dx, dy, lap, c;
};

template <int W>
__device__ __forceinline__ St2 stencil2(const float2* __restrict__ ring, int prv, int cur, int nxt, int s,
                                        bool want_lap) {
    const float2* A = ring + prv * W + s;
    const float2* B = ring + cur * W + s;
    const float2* C = ring + nxt * W + s;
    const v2 Bm = B[-1], Bc = B[0], Bp = B[1];
    const float* Af = reinterpret_cast<const float*>(A);
    const float* Cf = reinterpret_cast<const float*>(C);
    const v2 Sm = make_float2(Af[-1], Bm.x), Sc = make_float2(Af[1], Bc.x), Sp = make_float2(Af[3], Bp.x);
    const v2 Nm = make_float2(Bm.y, Cf[-2]), Nc = make_float2(Bc.y, Cf[0]), Np = make_float2(Bp.y, Cf[2]);
    St2 o;
    const v2 d1 = Np - Sm, d2 = Sp - Nm;  // NE - SW, SE - NW
    o.dx = fma2(Bp - Bm, bc(1.f / 3.f), (d1 + d2) * bc(1.f / 12.f));
    o.dy = fma2(Nc - Sc, bc(1.f / 3.f), (d1 - d2) * bc(1.f / 12.f));
    if (want_lap) {
        const v2 ax4 = (Bp + Bm) + (Nc + Sc);
        const v2 dg = (Np + Sm) + (Nm + Sp);
        o.lap = fma2(bc(-20.f), Bc, fma2(bc(4.f), ax4, dg)) * bc(1.f / 6.f);
    } else {
        o.lap = bc(0.f);
    }
    o.c = Bc;
    return o;
}

// K of Eq. 18 with per-cell coefficients (ax, ay, cA, cB) of the frozen flow:
// K = ax dT/dx + ay dT/dy + chi lap T - T (cA - cB phi'(T)),
// phi'(T) = k1^2 - k0 k1 / sqrt(T) (derivative of Eq. 21's phi).
__device__ __forceinline__ v2 rhs_K2(const St2& u, v2 ax, v2 ay, v2 cA, v2 cB, const StepParams& P) {
    const v2 T = u.c + bc(P.Ts);
    const v2 dphi = fma2(bc(-P.k0k1), rsqrt2(T), bc(P.k1k1));
    const v2 src = T * fma2(-cB, dphi, cA);
    return fma2(ax, u.dx, fma2(ay, u.dy, fma2(bc(P.chi), u.lap, -src)));
}

}  // namespace

template <int BD, int MINB>
__global__ void __launch_bounds__(BD, MINB) lb_step_pairs(const StepParams P) {
    constexpr int W = BD + 2;
    extern __shared__ float2 sm2[];
    __shared__ double red[BD / 32];
    float2* const sPSI = sm2;
    float2* const sRHO = sPSI + 4 * W;
    float2* const sVX = sRHO + 4 * W;
    float2* const sVY = sVX + 4 * W;
    float2* const sU2 = sVY + 4 * W;
    float2* const sU3 = sU2 + 4 * W;
    float2* const sU4 = sU3 + 4 * W;
    float2* const sTH = sU4 + 4 * W;  // 8 slots
    float2* const sCO = sTH + 8 * W;  // [4 coefficients][4 slots][BD], own column only
    for (int i = threadIdx.x; i < 36 * W + 16 * BD; i += BD) sm2[i] = make_float2(0.f, 0.f);

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
    const int ys = seg * P.seg_h;  // even
    const int ye = min(ys + P.seg_h, Ly);
    auto lo = [&](int d) { return periodic ? ys - d : max(ys - d, 0); };
    auto hi = [&](int d) { return periodic ? ye + d : min(ye + d, Ly); };
    const int loP = lo(5), hiP = hi(5), loB = lo(4), hiB = hi(4), loC = lo(3), hiC = hi(3);
    const int loD = lo(2), hiD = hi(2), loE = lo(1), hiE = hi(1);
    auto pin = [](int p, int l, int h) { return 2 * p + 1 >= l && 2 * p < h; };
    // wall rows (Dirichlet temperature, Zou-He populations, no force)
    auto wallrow = [&](int R) { return !periodic && (R == 0 || R == Ly - 1); };
    const bool thermal = !P.isothermal;
    bool eos_bad = false, nonfinite = false;

    const int q0 = (loP >= 0 ? loP : loP - 1) / 2;  // floor(loP / 2)
    const int q1 = (ye - 1 >= 0 ? (ye - 1) / 2 : -1) + 5;

    v2 fc[9], thc;
    load_pair(P, 2 * q0, x, xm, xp, fc, thc);
    v2 fP[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) fP[k] = bc(0.f);
    v2 accD = bc(0.f), accE = bc(0.f), accF = bc(0.f);
    __syncthreads();

    for (int q = q0; q <= q1; ++q) {
        // ---- P: wall fill, rho, psi of pair q
        if (pin(q, loP, hiP)) {
            const int R0 = 2 * q;
            if (!periodic) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int R = R0 + k;
                    float g[9];
#pragma unroll
                    for (int a = 0; a < 9; ++a) g[a] = k ? fc[a].y : fc[a].x;
                    if (R == 0 || R == Ly - 1) {
                        wall_fill(P, R, g);
#pragma unroll
                        for (int a = 0; a < 9; ++a) {
                            if (k) fc[a].y = g[a];
                            else fc[a].x = g[a];
                        }
                    }
                }
            }
            const v2 rho = ((fc[0] + fc[1]) + (fc[2] + fc[3])) + ((fc[4] + fc[5]) + (fc[6] + fc[7])) + fc[8];
            const v2 psi = eos_psi2(rho, thc + bc(P.Ts), P, eos_bad);
            sPSI[(q & 3) * W + s] = psi;
            sRHO[(q & 3) * W + s] = rho;
            sTH[(q & 7) * W + s] = thc;
        }
        __syncthreads();

        // ---- bottom-wall heat flux of level t (Sec. 3.2), one sample per step
        if (!periodic && ys == 0 && q == 1) {
            double qv = 0.0;
            if (outc) {
                const double r0 = sRHO[0 * W + s].x;
                const double t0 = sTH[0 * W + s].x, t1 = sTH[0 * W + s].y, t2 = sTH[1 * W + s].x;
                qv = -(double)P.cvchi * r0 * (-3.0 * t0 + 4.0 * t1 - t2) * 0.5;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) qv += __shfl_down_sync(0xffffffffu, qv, o);
            if ((lc & 31) == 0) red[lc >> 5] = qv;
            __syncthreads();
            if (lc == 0) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < BD / 32; ++w) sum += red[w];
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

        // ---- B: forces, velocity, collision of pair q-1
        {
            const int p = q - 1;
            if (pin(p, loB, hiB)) {
                const int R0 = 2 * p, R1 = R0 + 1;
                const int sl = (p & 3) * W + s;
                const v2 rho = sRHO[sl];
                const St2 g = stencil2<W>(sPSI, (p - 1) & 3, p & 3, (p + 1) & 3, s, false);
                v2 sx = g.dx, sy = g.dy;  // sum_a w_a psi(x + e_a) e_a, Eq. 7 (w = 1/3, 1/12)
                const v2 psi = g.c;
                const bool w0 = wallrow(R0), w1 = wallrow(R1);
                if (w0 | w1) {
                    // ghost-layer variant: the row beyond a wall copies the wall row
                    if (P.ghost) {
                        const float2* Bq = sPSI + (p & 3) * W + s;
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            const int R = R0 + k;
                            if (!wallrow(R)) continue;
                            const float2* rowc = Bq;
                            // psi rows below / at / above row R, with the ghost copy
                            float lo3[3], c3[3], hi3[3];
#pragma unroll
                            for (int d = -1; d <= 1; ++d) {
                                c3[d + 1] = k ? rowc[d].y : rowc[d].x;
                                const float below = k ? rowc[d].x : reinterpret_cast<const float*>(
                                                                        sPSI + ((p - 1) & 3) * W + s + d)[1];
                                const float above = k ? reinterpret_cast<const float*>(
                                                            sPSI + ((p + 1) & 3) * W + s + d)[0]
                                                      : rowc[d].y;
                                lo3[d + 1] = (R == 0) ? c3[d + 1] : below;
                                hi3[d + 1] = (R == Ly - 1) ? c3[d + 1] : above;
                            }
                            float gx, gy;
                            psi_sum(lo3 + 1, c3 + 1, hi3 + 1, gx, gy);
                            if (k) {
                                sx.y = gx;
                                sy.y = gy;
                            } else {
                                sx.x = gx;
                                sy.x = gy;
                            }
                        }
                    }
                }
                v2 Fmx = (-P.G) * (psi * sx), Fmy = (-P.G) * (psi * sy);
                const bool z0 = w0 && !P.ghost, z1 = w1 && !P.ghost;
                Fmx = sel(z0, z1, bc(0.f), Fmx);
                Fmy = sel(z0, z1, bc(0.f), Fmy);
                // F_b on fluid rows (Eq. 9); F_ads on the first fluid row (Eq. 22)
                v2 Fy = Fmy - sel(w0, w1, bc(0.f), P.g * (rho - bc(P.rho_ave)));
                if (!periodic && (R0 == 1 || R1 == 1)) {
                    const v2 ad = P.gw6 * (psi * psi);
                    Fy = Fy + sel(R0 == 1, R1 == 1, ad, bc(0.f));
                }
                const v2 Fx = Fmx;
                const v2 (&f)[9] = fP;
                const v2 jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
                const v2 jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
                const v2 irho = rcp2(rho);
                const v2 vx = fma2(bc(0.5f), Fx, jx) * irho;  // Eq. 6
                const v2 vy = fma2(bc(0.5f), Fy, jy) * irho;
                sVX[sl] = vx;
                sVY[sl] = vy;
                const bool st0 = outc && R0 >= ys && R0 < ye, st1 = outc && R1 >= ys && R1 < ye;
                if (st0 | st1) {
                    // MRT collision, Eq. 2 with S of Eq. 8, additive form f* = f + M^-1 dm
                    const v2 sa = (f[1] + f[3]) + (f[2] + f[4]);
                    const v2 sd = (f[5] + f[7]) + (f[6] + f[8]);
                    const v2 dxd = (f[5] - f[7]) + (f[8] - f[6]);
                    const v2 dyd = (f[5] - f[7]) + (f[6] - f[8]);
                    const v2 rv2 = rho * fma2(vx, vx, vy * vy);
                    const v2 ne1 = (fma2(bc(4.f), sd, sa) - 2.f * f[0]) - 3.f * rv2;
                    const v2 ne2 = 3.f * ((f[0] - sa) + rv2);
                    const v2 ne4 = fma2(bc(2.f), dxd, fma2(bc(0.5f), Fx, -(f[1] - f[3])));
                    const v2 ne6 = fma2(bc(2.f), dyd, fma2(bc(0.5f), Fy, -(f[2] - f[4])));
                    const v2 ne7 = ((f[1] + f[3]) - (f[2] + f[4])) - rho * fma2(vx, vx, -(vy * vy));
                    const v2 ne8 = ((f[5] + f[7]) - (f[6] + f[8])) - rho * (vx * vy);
                    const v2 vF = fma2(vx, Fx, vy * Fy);
                    const v2 psi2 = psi * psi;
                    const v2 fm2 = fma2(Fmx, Fmx, Fmy * Fmy);
                    const v2 ratio = make_float2(psi2.x > 0.f ? __fdividef(fm2.x, psi2.x) : 0.f,
                                                 psi2.y > 0.f ? __fdividef(fm2.y, psi2.y) : 0.f);
                    const v2 S1 = fma2(bc(6.f), vF, P.sig_e * ratio);
                    const v2 S2 = -fma2(bc(6.f), vF, P.sig_z * ratio);
                    const v2 S7 = 2.f * fma2(vx, Fx, -(vy * Fy));
                    const v2 S8 = fma2(vx, Fy, vy * Fx);
                    v2 sfr = (rho - bc(P.rho_v)) * bc(P.inv_drho);
                    sfr = make_float2(fminf(fmaxf(sfr.x, 0.f), 1.f), fminf(fmaxf(sfr.y, 0.f), 1.f));
                    const v2 snu = rcp2(fma2(bc(P.dtau), sfr, bc(P.tau_v)));
                    const v2 dm1 = fma2(bc(-P.s_e), ne1, (1.f - 0.5f * P.s_e) * S1);
                    const v2 dm2 = fma2(bc(-P.s_z), ne2, (1.f - 0.5f * P.s_z) * S2);
                    const v2 dm4 = fma2(bc(-P.s_q), ne4, (-(1.f - 0.5f * P.s_q)) * Fx);
                    const v2 dm6 = fma2(bc(-P.s_q), ne6, (-(1.f - 0.5f * P.s_q)) * Fy);
                    const v2 dm7 = fma2(-snu, ne7, fma2(bc(-0.5f), snu, bc(1.f)) * S7);
                    const v2 dm8 = fma2(-snu, ne8, fma2(bc(-0.5f), snu, bc(1.f)) * S8);
                    const v2 n1 = dm1 * bc(1.f / 36.f), n2 = dm2 * bc(1.f / 36.f);
                    const v2 n3 = Fx * bc(1.f / 6.f), n4 = dm4 * bc(1.f / 12.f);
                    const v2 n5 = Fy * bc(1.f / 6.f), n6 = dm6 * bc(1.f / 12.f);
                    const v2 n7 = dm7 * bc(0.25f), n8 = dm8 * bc(0.25f);
                    const v2 ax_ = fma2(bc(-2.f), n2, -n1);
                    const v2 dg = fma2(bc(2.f), n1, n2);
                    const v2 cx = fma2(bc(-2.f), n4, n3), cy = fma2(bc(-2.f), n6, n5);
                    const v2 dxx = n3 + n4, dyy = n5 + n6;
                    v2 o[9];
                    o[0] = fma2(bc(4.f), n2 - n1, f[0]);
                    o[1] = f[1] + ((ax_ + cx) + n7);
                    o[2] = f[2] + ((ax_ + cy) - n7);
                    o[3] = f[3] + ((ax_ - cx) + n7);
                    o[4] = f[4] + ((ax_ - cy) - n7);
                    o[5] = f[5] + ((dg + dxx) + (dyy + n8));
                    o[6] = f[6] + ((dg - dxx) + (dyy - n8));
                    o[7] = f[7] + ((dg - dxx) - (dyy - n8));
                    o[8] = f[8] + ((dg + dxx) - (dyy + n8));
                    const int pl = P.plane;
                    if (st0) {
                        if (!finite_f(rho.x)) nonfinite = true;
                        float* out = P.f_out + wrap(R0, Ly) * P.pitch + x;
#pragma unroll
                        for (int a = 0; a < 9; ++a) out[a * pl] = o[a].x;
                    }
                    if (st1) {
                        if (!finite_f(rho.y)) nonfinite = true;
                        float* out = P.f_out + wrap(R1, Ly) * P.pitch + x;
#pragma unroll
                        for (int a = 0; a < 9; ++a) out[a * pl] = o[a].y;
                    }
                }
            }
        }
        __syncthreads();

        // ---- the pulled populations of pair q+1 (consumed by P next iteration)
        v2 fn[9], thn = bc(0.f);
        if (pin(q + 1, loP, hiP)) {
            load_pair(P, 2 * q + 2, x, xm, xp, fn, thn);
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) fn[k] = bc(0.f);
        }

        v2 accC = bc(0.f);
        if (thermal) {
            // ---- C: frozen-flow coefficients and RK stage 1 of pair q-2
            {
                const int p = q - 2;
                if (pin(p, loC, hiC)) {
                    const int R0 = 2 * p, R1 = R0 + 1;
                    const int pm = (p - 1) & 3, pc = p & 3, pn = (p + 1) & 3;
                    const St2 gr = stencil2<W>(sRHO, pm, pc, pn, s, false);
                    const St2 gvx = stencil2<W>(sVX, pm, pc, pn, s, false);
                    const St2 gvy = stencil2<W>(sVY, pm, pc, pn, s, false);
                    const v2 rho = gr.c;
                    const v2 irho = rcp2(rho);
                    const v2 divv = gvx.dx + gvy.dy;
                    const v2 br = P.b * rho;
                    const v2 ax = fma2(bc(P.chi), gr.dx * irho, -gvx.c);
                    const v2 ay = fma2(bc(P.chi), gr.dy * irho, -gvy.c);
                    const v2 cA = (P.R * P.inv_cv) * divv * rcp2(bc(1.f) - br);
                    const v2 cB = (P.a * P.inv_cv) * (divv * rho) * rcp2(fma2(br, bc(2.f) - br, bc(1.f)));
                    sCO[(0 * 4 + pc) * BD + lc] = ax;
                    sCO[(1 * 4 + pc) * BD + lc] = ay;
                    sCO[(2 * 4 + pc) * BD + lc] = cA;
                    sCO[(3 * 4 + pc) * BD + lc] = cB;
                    const St2 ut = stencil2<W>(sTH, (p - 1) & 7, p & 7, (p + 1) & 7, s, true);
                    accC = rhs_K2(ut, ax, ay, cA, cB, P);
                    const bool w0 = wallrow(R0), w1 = wallrow(R1);
                    accC = sel(w0, w1, bc(0.f), accC);
                    sU2[pc * W + s] = fma2(bc(0.5f), accC, ut.c);
                }
            }
            __syncthreads();
            // ---- D: RK stage 2 of pair q-3
            {
                const int p = q - 3;
                if (pin(p, loD, hiD)) {
                    const int pc = p & 3;
                    const St2 u = stencil2<W>(sU2, (p - 1) & 3, pc, (p + 1) & 3, s, true);
                    v2 h = rhs_K2(u, sCO[(0 * 4 + pc) * BD + lc], sCO[(1 * 4 + pc) * BD + lc],
                                  sCO[(2 * 4 + pc) * BD + lc], sCO[(3 * 4 + pc) * BD + lc], P);
                    h = sel(wallrow(2 * p), wallrow(2 * p + 1), bc(0.f), h);
                    const v2 th = sTH[(p & 7) * W + s];
                    sU3[pc * W + s] = fma2(bc(0.5f), h, th);
                    accD = fma2(bc(2.f), h, accD);
                }
            }
            __syncthreads();
            // ---- E: RK stage 3 of pair q-4
            {
                const int p = q - 4;
                if (pin(p, loE, hiE)) {
                    const int pc = p & 3;
                    const St2 u = stencil2<W>(sU3, (p - 1) & 3, pc, (p + 1) & 3, s, true);
                    v2 h = rhs_K2(u, sCO[(0 * 4 + pc) * BD + lc], sCO[(1 * 4 + pc) * BD + lc],
                                  sCO[(2 * 4 + pc) * BD + lc], sCO[(3 * 4 + pc) * BD + lc], P);
                    h = sel(wallrow(2 * p), wallrow(2 * p + 1), bc(0.f), h);
                    const v2 th = sTH[(p & 7) * W + s];
                    sU4[pc * W + s] = th + h;
                    accE = fma2(bc(2.f), h, accE);
                }
            }
            __syncthreads();
        }
        // ---- F: RK stage 4 and theta^{t+1} of pair q-5
        {
            const int p = q - 5;
            const int R0 = 2 * p, R1 = R0 + 1;
            const bool st0 = outc && R0 >= ys && R0 < ye, st1 = outc && R1 >= ys && R1 < ye;
            if (st0 | st1) {
                const v2 th = sTH[(p & 7) * W + s];
                v2 tn = th;
                if (thermal) {
                    const int pc = p & 3;
                    const St2 u = stencil2<W>(sU4, (p - 1) & 3, pc, (p + 1) & 3, s, true);
                    const v2 h = rhs_K2(u, sCO[(0 * 4 + pc) * BD + lc], sCO[(1 * 4 + pc) * BD + lc],
                                        sCO[(2 * 4 + pc) * BD + lc], sCO[(3 * 4 + pc) * BD + lc], P);
                    tn = fma2(accF + h, bc(1.f / 6.f), th);
                    if (!periodic) {
                        const float tb = __ldg(P.thb + x);
                        if (R0 == 0) tn.x = tb;
                        if (R0 == Ly - 1) tn.x = 0.f;
                        if (R1 == Ly - 1) tn.y = 0.f;
                    }
                }
                if (st0) {
                    if (!finite_f(tn.x)) nonfinite = true;
                    P.th_out[wrap(R0, Ly) * P.pitch + x] = tn.x;
                }
                if (st1) {
                    if (!finite_f(tn.y)) nonfinite = true;
                    P.th_out[wrap(R1, Ly) * P.pitch + x] = tn.y;
                }
            }
        }
        // rotate carries
        accF = accE;
        accE = accD;
        accD = accC;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            fP[k] = fc[k];
            fc[k] = fn[k];
        }
        thc = thn;
    }
    if (eos_bad) atomicOr(&P.acc->err, ERR_EOS);
    if (nonfinite) atomicOr(&P.acc->err, ERR_NONFINITE);
}

namespace {

template <int BD, int MINB>
struct PairKernel {
    static size_t smem() { return sizeof(float2) * (size_t)(36 * (BD + 2) + 16 * BD); }
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(lb_step_pairs<BD, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem());
    }
    static cudaError_t occupancy(int* n) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lb_step_pairs<BD, MINB>, BD, smem());
    }
    static cudaError_t launch(const StepParams& P, int nblocks, cudaStream_t st) {
        lb_step_pairs<BD, MINB><<<nblocks, BD, smem(), st>>>(P);
        return cudaGetLastError();
    }
};

}  // namespace

// Block sizes of the paired kernel (threads per block); the host picks one.
bool pairs_supported(int block_x) { return block_x == 128 || block_x == 256; }

cudaError_t pairs_prepare() {
    cudaError_t e = PairKernel<128, 4>::prepare();
    if (e != cudaSuccess) return e;
    return PairKernel<256, 2>::prepare();
}

cudaError_t pairs_occupancy(int block_x, int* n) {
    if (block_x == 128) return PairKernel<128, 4>::occupancy(n);
    return PairKernel<256, 2>::occupancy(n);
}

cudaError_t pairs_launch(const StepParams& P, const Launch& L, cudaStream_t st) {
    const int nb = L.nstrips * L.nseg;
    if (L.block_x == 128) return PairKernel<128, 4>::launch(P, nb, st);
    return PairKernel<256, 2>::launch(P, nb, st);
}

}  // namespace lbgpu
