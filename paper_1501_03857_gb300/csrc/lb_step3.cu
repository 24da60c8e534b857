// The fused time step, one row per iteration, two column strips per block,
// with paired FP32 arithmetic.
//
// A block marches up a segment of rows through a pipeline of stages, each
// one row behind the previous; every population and temperature value is
// read from HBM once and written once per step. A block owns TWO adjacent column
// strips of (BD - 10) output columns each, and thread lc computes column lc
// of both; the two cells are packed in one float2 (strip A in .x, strip B in
// .y). A stencil neighbour of the pair is then again an aligned float2 in
// shared memory, and every row-level condition (walls, ghost layer, first
// fluid row) holds for both halves, so the whole update runs on Blackwell's
// paired FP32 instructions (__ffma2_rn / __fadd2_rn / __fmul2_rn: two FP32
// operations per issue slot) with no repacking. Barriers and ring indexing
// are shared by the two cells. Reciprocals and 1/sqrt are the special-
// function unit's approximations (PTX rcp.approx, rsqrt.approx: one
// instruction each, the values __fdividef(1, x) and rsqrtf give here, without
// their range handling); psi itself is correctly rounded (__fsqrt_rn).
//
//   P  row L    : pull f (loads issued one iteration ahead), wall fill,
//                 rho, psi(rho, T^t)                       (Eqs. 3, 6, 21)
//   B  row L-1  : F_m, F_ads, F_b, v, MRT collision, store f*   (Eqs. 2-9, 22)
//   C  row L-2  : grad rho, div v, RK stage 1 of Eq. 18        (Eqs. 18-20)
//   D  row L-3  : RK stage 2
//   E  row L-4  : RK stage 3
//   F  row L-5  : RK stage 4, store theta^{t+1}
#include "lb_internal.h"

#include <type_traits>

namespace lbgpu {

namespace {

// Two cells (strip A, strip B) in paired FP32: one __ffma2_rn / __fadd2_rn /
// __fmul2_rn does both.
struct P2 {
    float2 v;
    __device__ __forceinline__ P2() {}
    __device__ __forceinline__ explicit P2(float2 a) : v(a) {}
    __device__ __forceinline__ P2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ float x() const { return v.x; }
    __device__ __forceinline__ float y() const { return v.y; }
    __device__ __forceinline__ float2 f2() const { return v; }
    static __device__ __forceinline__ P2 bc(float s) { return P2(s, s); }
};
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2(__fadd2_rn(a.v, b.v)); }
// a - b is a paired add of -b: the negation is an operand modifier, so no
// (-1, -1) register pair has to be held for it
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ P2 operator-(P2 a) { return P2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ P2 operator*(float s, P2 b) { return P2(__fmul2_rn(make_float2(s, s), b.v)); }
__device__ __forceinline__ P2 fma2(P2 a, P2 b, P2 c) { return P2(__ffma2_rn(a.v, b.v, c.v)); }

// the special-function unit's approximate reciprocal and 1/sqrt (PTX
// rcp.approx / rsqrt.approx, flushing subnormals: none occur in the step)
__device__ __forceinline__ float rcp_approx(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float a) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
template <class T>
__device__ __forceinline__ T rcp2(T a) { return T(rcp_approx(a.x()), rcp_approx(a.y())); }
template <class T>
__device__ __forceinline__ T rsqrt2(T a) { return T(rsqrt_approx(a.x()), rsqrt_approx(a.y())); }

// y = v mod n for pipeline rows (|v| is within a few rows of [0, n)).
__device__ __forceinline__ int wrap_row(int v, int n) {
    if (v < 0) v += n;
    if (v >= n) v -= n;
    if ((unsigned)v >= (unsigned)n) v = wrap(v, n);
    return v;
}

// Pulled populations (Eq. 3: f_a(x) = f*_a(x - e_a)) and theta of row y for
// the two columns; sources beyond a wall read 0 (filled by Zou-He), with the
// outflow top the source row is clamped to the top row.
template <class T, bool CG>
__device__ __forceinline__ void load_row2(const StepParams& P, int y, int xa, int xam, int xap, int xb, int xbm,
                                          int xbp, T (&f)[9], T& th) {
    const float* __restrict__ F = P.f_in;
    const int pl = P.plane, pitch = P.pitch;
    const size_t nF = 9 * (size_t)pl;
    int ym = y - 1, yp = y + 1;
    bool okm = true, okp = true;
    if (P.bc == BC_PERIODIC) {
        if (ym < 0) ym += P.Ly;
        if (yp >= P.Ly) yp -= P.Ly;
    } else {
        okm = ym >= 0;
        if (yp >= P.Ly) {
            if (P.bc == BC_TOP_OUTFLOW) yp = P.Ly - 1;
            else okp = false;
        }
    }
    const float* Rc = F + y * pitch;
    const float* Rm = F + ym * pitch;
    const float* Rp = F + yp * pitch;
    f[0] = T(lb_ld<CG>(Rc + xa, F, nF, P.acc), lb_ld<CG>(Rc + xb, F, nF, P.acc));
    f[1] = T(lb_ld<CG>(Rc + pl + xam, F, nF, P.acc), lb_ld<CG>(Rc + pl + xbm, F, nF, P.acc));
    f[3] = T(lb_ld<CG>(Rc + 3 * pl + xap, F, nF, P.acc), lb_ld<CG>(Rc + 3 * pl + xbp, F, nF, P.acc));
    if (okm) {
        f[2] = T(lb_ld<CG>(Rm + 2 * pl + xa, F, nF, P.acc), lb_ld<CG>(Rm + 2 * pl + xb, F, nF, P.acc));
        f[5] = T(lb_ld<CG>(Rm + 5 * pl + xam, F, nF, P.acc), lb_ld<CG>(Rm + 5 * pl + xbm, F, nF, P.acc));
        f[6] = T(lb_ld<CG>(Rm + 6 * pl + xap, F, nF, P.acc), lb_ld<CG>(Rm + 6 * pl + xbp, F, nF, P.acc));
    } else {
        f[2] = f[5] = f[6] = T::bc(0.f);
    }
    if (okp) {
        f[4] = T(lb_ld<CG>(Rp + 4 * pl + xa, F, nF, P.acc), lb_ld<CG>(Rp + 4 * pl + xb, F, nF, P.acc));
        f[7] = T(lb_ld<CG>(Rp + 7 * pl + xap, F, nF, P.acc), lb_ld<CG>(Rp + 7 * pl + xbp, F, nF, P.acc));
        f[8] = T(lb_ld<CG>(Rp + 8 * pl + xam, F, nF, P.acc), lb_ld<CG>(Rp + 8 * pl + xbm, F, nF, P.acc));
    } else {
        f[4] = f[7] = f[8] = T::bc(0.f);
    }
    const float* Tc = P.th_in + y * pitch;
    th = T(lb_ld<CG>(Tc + xa, P.th_in, (size_t)pl, P.acc), lb_ld<CG>(Tc + xb, P.th_in, (size_t)pl, P.acc));
}

// Isotropic central differences (Lee and Lin; Sec. 2 after Eq. 20) at
// column s, rows m (below), c, p (above) of float2 ring rows, without their
// common factors: dx, dy are 12 x the first derivatives (weights 1/3 axis,
// 1/12 diagonal: the same as sum_a w_a phi(x + e_a) e_a of Eq. 7) and lap is
// 6 x the laplacian. The factors are folded into the per-row coefficients
// that multiply them.
template <class T>
struct St2 {
    T dx, dy, lap, c;
};

template <class T>
__device__ __forceinline__ St2<T> stencil2(const float2* __restrict__ m, const float2* __restrict__ c,
                                           const float2* __restrict__ p, bool want_lap) {
    const T W(c[-1]), C(c[0]), E(c[1]);
    const T SW(m[-1]), S(m[0]), SE(m[1]);
    const T NW(p[-1]), N(p[0]), NE(p[1]);
    const T d1 = NE - SW, d2 = SE - NW;
    St2<T> o;
    o.dx = fma2(T::bc(4.f), E - W, d1 + d2);
    o.dy = fma2(T::bc(4.f), N - S, d1 - d2);
    if (want_lap) {
        const T ax4 = (E + W) + (N + S);
        const T dg = (NE + SW) + (NW + SE);
        o.lap = fma2(T::bc(-20.f), C, fma2(T::bc(4.f), ax4, dg));
    } else {
        o.lap = T::bc(0.f);
    }
    o.c = C;
    return o;
}

// Per-cell coefficients of K(T), Eq. 18, with rho and v frozen at level t:
// K = ax dT/dx + ay dT/dy + chi lap T - T (cA - cB phi'(T)), where
// ax = -v_x + chi d_x rho / rho (div(lambda grad T)/(rho c_v) with
// lambda = c_v chi rho), cA - cB phi' = (dp/dT)_rho div v / (rho c_v) and
// phi'(T) = k1^2 - k0 k1 / sqrt(T) (derivative of Eq. 21's phi). ax and ay
// are stored divided by 12 (they multiply the unweighted stencil sums).
template <class T>
struct Coef2 {
    T ax, ay, cA, cB;
};

template <class T>
__device__ __forceinline__ T rhs_K2(const St2<T>& u, const Coef2<T>& k, const StepParams& P) {
    const T Tt = u.c + T(P.kp[KP_TS]);
    const T dphi = fma2(T(P.kp[KP_K0K1N]), rsqrt2(Tt), T(P.kp[KP_K1K1]));
    const T src = Tt * fma2(-k.cB, dphi, k.cA);
    return fma2(k.ax, u.dx, fma2(k.ay, u.dy, fma2(T(P.kp[KP_CHI6]), u.lap, -src)));
}

// psi of Sec. 2 with the Peng-Robinson EOS of Eq. 21 for two cells.
template <class T>
__device__ __forceinline__ T eos_psi2(T rho, T Tt, const StepParams& P, bool& bad) {
    const T sT = Tt * rsqrt2(Tt);
    T ph = fma2(T(P.kp[KP_K1N]), sT, T(P.kp[KP_K0]));
    ph = ph * ph;
    // p = R rho T / d1 - a phi rho^2 / d2 over the common denominator d1 d2
    const T br = T(P.kp[KP_B]) * rho;
    const T d1 = T::bc(1.f) - br;
    const T d2 = fma2(br, T::bc(2.f) - br, T::bc(1.f));  // 1 + 2 b rho - b^2 rho^2
    const T p = fma2((T(P.kp[KP_R]) * rho) * Tt, d2, -(((T(P.kp[KP_A]) * ph) * (rho * rho)) * d1)) * rcp2(d1 * d2);
    const T arg = T(P.kp[KP_2G]) * fma2(rho, T::bc(-1.f / 3.f), p);
    const float ax = arg.x(), ay = arg.y();
    bad |= (ax < 0.f) | (ay < 0.f);
    // correctly rounded: psi multiplies the neighbour sums of Eq. 7, so its
    // relative error reaches the velocity amplified by |F_m| / (rho |v|)
    return T(__fsqrt_rn(fmaxf(ax, 0.f)), __fsqrt_rn(fmaxf(ay, 0.f)));
}

// MRT collision, Eq. 2 with the forcing moments S of Eq. 8, in the exactly
// equivalent additive form f* = f + M^-1 dm, dm = -Lambda (m - m^eq) +
// (I - Lambda/2) S, for two cells. dm is small (non-equilibrium moments and
// forces), so FP32 rounding stays at ~1 ulp of f and dm_rho = 0 conserves
// mass exactly; the non-equilibrium moments use rho v = j + F/2 (Eq. 6).
// g2 = 144 |sum_a w_a psi(x + e_a) e_a|^2: with F_m = -G psi sum_a ... of
// Eq. 7, the |F_m|^2 / psi^2 of the sigma term of Eq. 8 is G^2 g2 / 144.
template <class T>
__device__ __forceinline__ void collide2(const T (&f)[9], T rho, T vx, T vy, T Fx, T Fy, T g2,
                                         const StepParams& P, T (&o)[9]) {
    const T sa = (f[1] + f[3]) + (f[2] + f[4]);
    const T sd = (f[5] + f[7]) + (f[6] + f[8]);
    const T dxd = (f[5] - f[7]) + (f[8] - f[6]);
    const T dyd = (f[5] - f[7]) + (f[6] - f[8]);
    const T rv2 = rho * fma2(vx, vx, vy * vy);
    const T ne1 = fma2(T::bc(-2.f), f[0], fma2(T::bc(4.f), sd, sa)) - 3.f * rv2;
    const T ne2t = (f[0] - sa) + rv2;  // (epsilon - epsilon^eq) / 3
    const T ne7 = ((f[1] + f[3]) - (f[2] + f[4])) - rho * fma2(vx, vx, -(vy * vy));
    const T ne8 = ((f[5] + f[7]) - (f[6] + f[8])) - rho * (vx * vy);
    const T vF = fma2(vx, Fx, vy * Fy);
    const T S7 = 2.f * fma2(vx, Fx, -(vy * Fy));
    const T S8 = fma2(vx, Fy, vy * Fx);
    // tau_nu(rho): linear between the coexistence densities, clamped to [0, 1]
    const float sr0 = -P.rho_v * P.inv_drho;
    const T sfr(__saturatef(fmaf(rho.x(), P.inv_drho, sr0)), __saturatef(fmaf(rho.y(), P.inv_drho, sr0)));
    // M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) applied
    // to dm (dm_j = F): n_k = dm_k times its diagonal entry, the entry folded
    // into the relaxation constants. dm_e, dm_eps: rates s_e, s_z with the
    // sigma source S = +-(6 v.F + sigma' |F_m|^2 / psi^2) (Eq. 8).
    const T n1 = fma2(T(P.kp[KP_SE36N]), ne1, fma2(T(P.kp[KP_KE6]), vF, T(P.kp[KP_KESIG]) * g2));
    const T n2 = fma2(T(P.kp[KP_SZ12N]), ne2t, fma2(T(P.kp[KP_KZ6N]), vF, T(P.kp[KP_KZSIGN]) * g2));
    // dm_q = -s_q (q - q^eq) + (s_q/2 - 1) F with q - q^eq = qh + F/2, so
    // dm_q = -s_q qh - F; with n3 = F_x/6, n4 = dm_qx/12: n3 - 2 n4 =
    // F_x/3 + (s_q/6) qh_x and n3 + n4 = F_x/12 - (s_q/12) qh_x
    const T qhx = fma2(T::bc(2.f), dxd, f[3] - f[1]);
    const T qhy = fma2(T::bc(2.f), dyd, f[4] - f[2]);
    const T cx = fma2(T(P.kp[KP_SQ6]), qhx, T::bc(1.f / 3.f) * Fx);
    const T cy = fma2(T(P.kp[KP_SQ6]), qhy, T::bc(1.f / 3.f) * Fy);
    const T dxx = fma2(T(P.kp[KP_SQ12N]), qhx, T::bc(1.f / 12.f) * Fx);
    const T dyy = fma2(T(P.kp[KP_SQ12N]), qhy, T::bc(1.f / 12.f) * Fy);
    // p_xx, p_xy: rate s_nu(rho), quartered: snu4 = s_nu / 4, hnu4 = (1 - s_nu/2) / 4
    const T snu4 = rcp2(fma2(T(P.kp[KP_DTAU4]), sfr, T(P.kp[KP_TAUV4])));
    const T hnu4 = fma2(T::bc(-0.5f), snu4, T::bc(0.25f));
    const T n7 = fma2(-snu4, ne7, hnu4 * S7);
    const T n8 = fma2(-snu4, ne8, hnu4 * S8);
    const T ax_ = fma2(T::bc(-2.f), n2, -n1);
    const T dg = fma2(T::bc(2.f), n1, n2);
    o[0] = fma2(T::bc(4.f), n2 - n1, f[0]);
    o[1] = f[1] + ((ax_ + cx) + n7);
    o[2] = f[2] + ((ax_ + cy) - n7);
    o[3] = f[3] + ((ax_ - cx) + n7);
    o[4] = f[4] + ((ax_ - cy) - n7);
    o[5] = f[5] + ((dg + dxx) + (dyy + n8));
    o[6] = f[6] + ((dg - dxx) + (dyy - n8));
    o[7] = f[7] + ((dg - dxx) - (dyy - n8));
    o[8] = f[8] + ((dg + dxx) - (dyy + n8));
}

}  // namespace

// The whole step for block `block` of the launch described by P. K supplies
// the model constants (kp except the wettability and rho_ave pairs,
// inv_drho, rho_v, cvchi): the same struct as P for one domain, or the
// batch's shared constants in the parameter bank while P is an instance's
// copy in shared memory. With REC (the adjoint's recompute mode) the block
// writes the forward intermediates of its own cells to R (RecomputeOut,
// lb_internal.h); with OUT it writes the collided populations and
// theta^{t+1}; with QF it adds q(t) to the heat-flux sums. The plain step is
// OUT and QF; the adjoint's replay of a checkpoint segment REC and OUT; its
// forward pass when it stores every step REC, OUT and QF.
template <int BD, class T, bool REC = false, bool CG = false, bool OUT = !REC, bool QF = !REC>
__device__ __forceinline__ void step_body(const StepParams& P, const StepParams& K, const int block,
                                          const RecomputeOut* R = nullptr) {
    constexpr int W = BD + 2;
    extern __shared__ float2 sm2[];
    __shared__ double red[BD / 32];
    float2* const sPSI = sm2;
    float2* const sRHO = sPSI + RING * W;
    float2* const sVX = sRHO + RING * W;
    float2* const sVY = sVX + RING * W;
    float2* const sU2 = sVY + RING * W;
    float2* const sU3 = sU2 + RING * W;
    float2* const sU4 = sU3 + RING * W;
    float2* const sTH = sU4 + RING * W;   // TRING slots
    float2* const sCO = sTH + TRING * W;  // [4 coefficients][RING slots][BD], own column
    constexpr size_t SMN = (size_t)SM_ROWS * W + 4 * RING * BD;  // float2 in the dynamic shared memory
    for (int i = threadIdx.x; i < (int)SMN; i += BD) sm2[i] = make_float2(0.f, 0.f);
    // checked build: a ring cell with its two x neighbours (smp), or a
    // coefficient slot with its three siblings (smc), inside the shared array
#ifdef LB_CHECKED
    auto smp = [&](auto* q) {
        if (q - 1 >= sm2 && q + 1 < sm2 + SMN) return q;
        atomicOr(&P.acc->err, ERR_BOUNDS);
        return static_cast<decltype(q)>(sm2 + 1);
    };
    auto smc = [&](auto* q) {
        if (q >= sm2 && q + 3 * RING * BD < sm2 + SMN) return q;
        atomicOr(&P.acc->err, ERR_BOUNDS);
        return static_cast<decltype(q)>(sm2);
    };
#define LB_SMP(q) smp(q)
#define LB_SMC(q) smc(q)
#else
#define LB_SMP(q) (q)
#define LB_SMC(q) (q)
#endif

    const int Lx = P.Lx, Ly = P.Ly;
    const int strip = block % P.nstrips;  // a pair of column strips
    const int seg = block / P.nstrips;
    const int nout = P.nout;
    const int x0 = strip * 2 * nout;
    const int nva = min(nout, Lx - x0);
    const int nvb = min(nout, Lx - x0 - nout);
    const int lc = threadIdx.x;
    const int s = lc + 1;
    const int xa = wrap(x0 - HALO + lc, Lx);
    const int xb = wrap(x0 + nout - HALO + lc, Lx);
    const int xam = xa == 0 ? Lx - 1 : xa - 1, xap = xa == Lx - 1 ? 0 : xa + 1;
    const int xbm = xb == 0 ? Lx - 1 : xb - 1, xbp = xb == Lx - 1 ? 0 : xb + 1;
    const bool outa = lc >= HALO && lc < HALO + nva;
    const bool outb = lc >= HALO && lc < HALO + nvb;
    const bool periodic = P.bc == BC_PERIODIC;
    const int ys = seg * P.seg_h;
    const int ye = min(ys + P.seg_h, Ly);
    auto lo = [&](int d) { return periodic ? ys - d : max(ys - d, 0); };
    // with walls every pipeline row is in [0, Ly) and is its own physical row
    auto interior = [&](int r) { return periodic || (r != 0 && r != Ly - 1); };
    auto hi = [&](int d) { return periodic ? ye + d : min(ye + d, Ly); };
    const int loP = lo(5), hiP = hi(5), loB = lo(4), hiB = hi(4), loC = lo(3), hiC = hi(3);
    const int loD = lo(2), hiD = hi(2), loE = lo(1), hiE = hi(1);
    const bool thermal = !P.isothermal;
    bool eos_bad = false, nonfinite = false;
    // recompute mode: a value pair into row y of a pitched plane, own columns
    auto put = [&](float* plane, int y, T v) {
        float* row = plane + y * P.pitch;
        if (outa) lb_st(row + xa, v.x(), plane, (size_t)P.plane, P.acc);
        if (outb) lb_st(row + xb, v.y(), plane, (size_t)P.plane, P.acc);
    };
    const T zero = T::bc(0.f);

    T fc[9], tc = zero;
    if (loP < hiP) load_row2<T, CG>(P, wrap_row(loP, Ly), xa, xam, xap, xb, xbm, xbp, fc, tc);
    T fP[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) fP[a] = zero;
    T acc1 = zero, acc2 = zero, acc3 = zero;
    // the RK coefficients of row r live in slot (r & 3) of sCO
    auto coef = [&](int r) {
        const float2* c = LB_SMC(sCO + (r & 3) * BD + lc);
        return Coef2<T>{T(c[0]), T(c[RING * BD]), T(c[2 * RING * BD]), T(c[3 * RING * BD])};
    };
    __syncthreads();

    int yL = wrap_row(loP, Ly);  // physical row of pipeline row L
    // One iteration of the pipeline. In the steady part (S) every stage's row
    // lies in the block's own rows and off the walls, so the range and wall
    // tests are compiled out; the first and last iterations keep them.
    auto iter = [&](const int L, auto steady) {
        constexpr bool S = decltype(steady)::value;
        // ---- prefetch the pulled populations of row L+1
        T fn[9], tn = zero;
        const int yN = yL + 1 == Ly ? 0 : yL + 1;
        // (the range test stays in the steady part too: without it the
        // loads are no longer issued a whole iteration ahead of their use,
        // and their latency shows up as long-scoreboard stalls, 1.3 cycles
        // per issued instruction instead of 0.2)
        if (L + 1 < hiP) {
            load_row2<T, CG>(P, yN, xa, xam, xap, xb, xbm, xbp, fn, tn);
        } else {
#pragma unroll
            for (int a = 0; a < 9; ++a) fn[a] = zero;
        }

        // ---- P: wall fill, rho, psi of row L
        if (S || L < hiP) {
            const int y = yL;
            if (!S && !periodic && y == 0) {  // Zou-He bottom wall, u = 0
                const T d = 0.5f * (fc[1] - fc[3]);
                fc[2] = fc[4];
                fc[5] = fc[7] - d;
                fc[6] = fc[8] + d;
            }
            if (!S && P.bc == BC_WALLS && y == Ly - 1) {  // Zou-He top wall, u = 0
                const T d = 0.5f * (fc[1] - fc[3]);
                fc[4] = fc[2];
                fc[7] = fc[5] + d;
                fc[8] = fc[6] - d;
            }
            const T rhoN = ((fc[0] + fc[1]) + (fc[2] + fc[3])) + ((fc[4] + fc[5]) + (fc[6] + fc[7])) + fc[8];
            const T psiN = eos_psi2(rhoN, tc + T(K.kp[KP_TS]), K, eos_bad);
            *LB_SMP(sPSI + (L & 3) * W + s) = psiN.f2();
            *LB_SMP(sRHO + (L & 3) * W + s) = rhoN.f2();
            *LB_SMP(sTH + (L & 7) * W + s) = tc.f2();
            if constexpr (REC) {
                if (L >= ys && L < ye) {
                    put(R->rho, y, rhoN);
                    put(R->psi, y, psiN);
                }
            }
        }
        __syncthreads();

        // ---- bottom-wall heat flux of level t (Sec. 3.2), one sample per step
        if (QF && !S && !periodic && ys == 0 && L == 2) {
            double qv = 0.0;
            const float2 r0 = *LB_SMP(sRHO + 0 * W + s), t0 = *LB_SMP(sTH + 0 * W + s), t1 = *LB_SMP(sTH + 1 * W + s), t2 = *LB_SMP(sTH + 2 * W + s);
            if (outa) qv += -(double)K.cvchi * r0.x * (-3.0 * t0.x + 4.0 * t1.x - t2.x) * 0.5;
            if (outb) qv += -(double)K.cvchi * r0.y * (-3.0 * t0.y + 4.0 * t1.y - t2.y) * 0.5;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) qv += __shfl_down_sync(0xffffffffu, qv, o);
            if ((lc & 31) == 0) red[lc >> 5] = qv;
            __syncthreads();
            // each strip's sum goes to its own slot (folded at the block's end)
            if (lc == 0) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < BD / 32; ++w) sum += red[w];
                P.qpart[strip] = sum;
            }
        }

        // ---- B: forces, velocity, collision of row L-1
        {
            const int r = L - 1;
            if (S || (r >= loB && r < hiB)) {
                const int y = yL == 0 ? Ly - 1 : yL - 1;
                const bool wall = !S && !periodic && (y == 0 || y == Ly - 1);
                const T rhoP(*LB_SMP(sRHO + (r & 3) * W + s));
                const T psiP(*LB_SMP(sPSI + (r & 3) * W + s));
                const T jxP = (fP[1] - fP[3]) + (fP[5] - fP[6]) + (fP[8] - fP[7]);
                const T jyP = (fP[2] - fP[4]) + (fP[5] + fP[6]) - (fP[7] + fP[8]);
                T Fmx = zero, Fmy = zero, g2 = zero;
                if (!wall || P.ghost) {
                    const float2* pc = sPSI + (r & 3) * W + s;
                    const float2* pn = (wall && y == Ly - 1) ? pc : sPSI + ((r + 1) & 3) * W + s;
                    const float2* ps = (wall && y == 0) ? pc : sPSI + ((r - 1) & 3) * W + s;
                    const St2<T> g = stencil2<T>(LB_SMP(ps), LB_SMP(pc), LB_SMP(pn), false);  // 12 sum_a w_a psi(x + e_a) e_a, Eq. 7
                    const T mG = T(K.kp[KP_GN12]) * psiP;
                    Fmx = mG * g.dx;
                    Fmy = mG * g.dy;
                    g2 = fma2(g.dx, g.dx, g.dy * g.dy);
                }
                T Fy = Fmy;
                if (!wall) {
                    if (!S && !periodic && y == 1) Fy = fma2(T(P.kp[KP_GW6]), psiP * psiP, Fy);  // Eq. 22
                    Fy = fma2(T(K.kp[KP_GN]), rhoP - T(P.kp[KP_RHOAVE]), Fy);                // Eq. 9
                }
                const T Fx = Fmx;
                const T irho = rcp2(rhoP);
                const T vx = fma2(T::bc(0.5f), Fx, jxP) * irho;  // Eq. 6
                const T vy = fma2(T::bc(0.5f), Fy, jyP) * irho;
                *LB_SMP(sVX + (r & 3) * W + s) = vx.f2();
                *LB_SMP(sVY + (r & 3) * W + s) = vy.f2();
                const bool st = S || (r >= ys && r < ye);
                if (OUT && st && (outa || outb)) {
                    T o[9];
                    collide2(fP, rhoP, vx, vy, Fx, Fy, g2, K, o);
                    const int pl = P.plane;
                    float* out = P.f_out + y * P.pitch;
                    if (outa) {
                        if (!finite_f(rhoP.x())) nonfinite = true;
#pragma unroll
                        for (int a = 0; a < 9; ++a) lb_st(out + (a * pl + xa), o[a].x(), P.f_out, 9 * (size_t)pl, P.acc);
                    }
                    if (outb) {
                        if (!finite_f(rhoP.y())) nonfinite = true;
#pragma unroll
                        for (int a = 0; a < 9; ++a) lb_st(out + (a * pl + xb), o[a].y(), P.f_out, 9 * (size_t)pl, P.acc);
                    }
                }
            }
        }
        __syncthreads();

        // Stage C makes the coefficients of row L-2 (kept in sCO); D, E, F work
        // on rows whose coefficients C made 1, 2 and 3 iterations ago.
        T accC = zero;
        if (thermal) {
            // ---- C: frozen-flow coefficients and RK stage 1 of row L-2
            {
                const int r = L - 2;
                if (S || (r >= loC && r < hiC)) {
                    const T thr(*LB_SMP(sTH + (r & 7) * W + s));
                    T u2 = thr;
                    if (S || interior(r)) {
                        const int om = ((r - 1) & 3) * W + s, oc = (r & 3) * W + s, op = ((r + 1) & 3) * W + s;
                        const St2<T> gr = stencil2<T>(LB_SMP(sRHO + om), LB_SMP(sRHO + oc), LB_SMP(sRHO + op), false);
                        const St2<T> gvx = stencil2<T>(LB_SMP(sVX + om), LB_SMP(sVX + oc), LB_SMP(sVX + op), false);
                        const St2<T> gvy = stencil2<T>(LB_SMP(sVY + om), LB_SMP(sVY + oc), LB_SMP(sVY + op), false);
                        const T rho = gr.c;
                        const T q = T(K.kp[KP_CHI144]) * rcp2(rho);
                        const T divv = gvx.dx + gvy.dy;  // 12 div v
                        const T br = T(K.kp[KP_B]) * rho;
                        Coef2<T> kC;  // ax, ay divided by 12
                        kC.ax = fma2(q, gr.dx, T::bc(-1.f / 12.f) * gvx.c);
                        kC.ay = fma2(q, gr.dy, T::bc(-1.f / 12.f) * gvy.c);
                        kC.cA = T(K.kp[KP_RCV12]) * divv * rcp2(T::bc(1.f) - br);
                        kC.cB = T(K.kp[KP_ACV12]) * (divv * rho) * rcp2(fma2(br, T::bc(2.f) - br, T::bc(1.f)));
                        float2* c = LB_SMC(sCO + (r & 3) * BD + lc);
                        c[0] = kC.ax.f2();
                        c[RING * BD] = kC.ay.f2();
                        c[2 * RING * BD] = kC.cA.f2();
                        c[3 * RING * BD] = kC.cB.f2();
                        const St2<T> ut = stencil2<T>(LB_SMP(sTH + ((r - 1) & 7) * W + s), LB_SMP(sTH + (r & 7) * W + s), LB_SMP(sTH + ((r + 1) & 7) * W + s), true);
                        accC = rhs_K2(ut, kC, K);
                        u2 = fma2(T::bc(0.5f), accC, thr);
                        if constexpr (REC) {
                            if (S || (r >= ys && r < ye)) {  // weighted gradients, unscaled coefficients
                                const int y = periodic ? wrap_row(yL - 2, Ly) : r;
                                const T w12 = T::bc(1.f / 12.f), t12 = T::bc(12.f);
                                put(R->drx, y, w12 * gr.dx);
                                put(R->dry, y, w12 * gr.dy);
                                put(R->divv, y, w12 * divv);
                                put(R->ax, y, t12 * kC.ax);
                                put(R->ay, y, t12 * kC.ay);
                            }
                        }
                    } else if constexpr (REC) {
                        if (r >= ys && r < ye) {
                            const int y = periodic ? wrap_row(yL - 2, Ly) : r;
                            put(R->drx, y, zero);
                            put(R->dry, y, zero);
                            put(R->divv, y, zero);
                            put(R->ax, y, zero);
                            put(R->ay, y, zero);
                        }
                    }
                    *LB_SMP(sU2 + (r & 3) * W + s) = u2.f2();
                    if constexpr (REC) {
                        if (S || (r >= ys && r < ye)) put(R->u2, periodic ? wrap_row(yL - 2, Ly) : r, u2);
                    }
                }
            }
            __syncthreads();
            // ---- D: RK stage 2 of row L-3
            {
                const int r = L - 3;
                if (S || (r >= loD && r < hiD)) {
                    const T thr(*LB_SMP(sTH + (r & 7) * W + s));
                    T u3 = thr;
                    if (S || interior(r)) {
                        const St2<T> u = stencil2<T>(LB_SMP(sU2 + ((r - 1) & 3) * W + s), LB_SMP(sU2 + (r & 3) * W + s), LB_SMP(sU2 + ((r + 1) & 3) * W + s), true);
                        const T h2 = rhs_K2(u, coef(r), K);
                        u3 = fma2(T::bc(0.5f), h2, thr);
                        acc1 = fma2(T::bc(2.f), h2, acc1);
                    }
                    *LB_SMP(sU3 + (r & 3) * W + s) = u3.f2();
                    if constexpr (REC) {
                        if (S || (r >= ys && r < ye)) put(R->u3, periodic ? wrap_row(yL - 3, Ly) : r, u3);
                    }
                }
            }
            __syncthreads();
            // ---- E: RK stage 3 of row L-4
            {
                const int r = L - 4;
                if (S || (r >= loE && r < hiE)) {
                    const T thr(*LB_SMP(sTH + (r & 7) * W + s));
                    T u4 = thr;
                    if (S || interior(r)) {
                        const St2<T> u = stencil2<T>(LB_SMP(sU3 + ((r - 1) & 3) * W + s), LB_SMP(sU3 + (r & 3) * W + s), LB_SMP(sU3 + ((r + 1) & 3) * W + s), true);
                        const T h3 = rhs_K2(u, coef(r), K);
                        u4 = thr + h3;
                        acc2 = fma2(T::bc(2.f), h3, acc2);
                    }
                    *LB_SMP(sU4 + (r & 3) * W + s) = u4.f2();
                    if constexpr (REC) {
                        if (S || (r >= ys && r < ye)) put(R->u4, periodic ? wrap_row(yL - 4, Ly) : r, u4);
                    }
                }
            }
            __syncthreads();
        }
        // ---- F: RK stage 4 and theta^{t+1} of row L-5
        {
            const int r = L - 5;
            if (OUT && (S || (r >= ys && r < ye)) && (outa || outb)) {
                const int y = periodic ? wrap_row(yL - 5, Ly) : r;
                const T thr(*LB_SMP(sTH + (r & 7) * W + s));
                T tnew = thr;
                if (thermal) {
                    if (!S && !periodic && y == 0) {
                        tnew = T(lb_ldg(P.thb + xa, P.thb, P.pitch, P.acc), lb_ldg(P.thb + xb, P.thb, P.pitch, P.acc));
                    } else if (!S && !periodic && y == Ly - 1) {
                        tnew = zero;
                    } else {
                        const St2<T> u = stencil2<T>(LB_SMP(sU4 + ((r - 1) & 3) * W + s), LB_SMP(sU4 + (r & 3) * W + s), LB_SMP(sU4 + ((r + 1) & 3) * W + s), true);
                        const T h4 = rhs_K2(u, coef(r), K);
                        tnew = fma2(acc3 + h4, T::bc(1.f / 6.f), thr);
                    }
                }
                float* out = P.th_out + y * P.pitch;
                if (outa) {
                    if (!finite_f(tnew.x())) nonfinite = true;
                    lb_st(out + xa, tnew.x(), P.th_out, (size_t)P.plane, P.acc);
                }
                if (outb) {
                    if (!finite_f(tnew.y())) nonfinite = true;
                    lb_st(out + xb, tnew.y(), P.th_out, (size_t)P.plane, P.acc);
                }
            }
        }
        // rotate per-thread carries
        acc3 = acc2;
        acc2 = acc1;
        acc1 = accC;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            fP[a] = fc[a];
            fc[a] = fn[a];
        }
        tc = tn;
        yL = yN;
    };
    // steady iterations: F's row L-5 >= ys (B, C, D, E then also in the
    // block's rows), B's row L-1 < ye; with walls F's row >= 1 and P's row
    // L <= Ly - 2, so no stage meets a wall row or the first fluid row
    const int Ls = ys + 5 + (!periodic && ys == 0 ? 1 : 0);
    const int Le = max(Ls, periodic ? ye + 1 : min(ye + 1, Ly - 1));
    int L = loP;
    for (; L < Ls; ++L) iter(L, std::false_type{});
    for (; L < Le; ++L) iter(L, std::true_type{});
    for (; L <= ye + 4; ++L) iter(L, std::false_type{});
    if (eos_bad) atomicOr(&P.acc->err, ERR_EOS);
    if (nonfinite) atomicOr(&P.acc->err, ERR_NONFINITE);
    // the strip that finishes last among the bottom segment's folds the slots
    // in strip order into q(t), so q(t) does not depend on the order in which
    // the blocks finish (folding here, when the block has no work left,
    // costs nothing; folding right after the partial sums delayed that block
    // and lengthened the step by 4 %)
    if (QF && !periodic && ys == 0) {
        __shared__ bool s_last;
        if (lc == 0) {
            __threadfence();
            s_last = atomicAdd(&P.acc->count, 1u) == (unsigned)P.nstrips - 1u;
        }
        __syncthreads();
        if (s_last && lc < 32) {
            __threadfence();
            double tot = 0.0;
            for (int k = lc; k < P.nstrips; k += 32) tot += __ldcg(P.qpart + k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            if (lc == 0) {
                // the sums are read and written at L2: in the persistent
                // batch another SM may hold an old copy of them in its L1
                Acc* A = P.acc;
                const double qt = tot / (double)Lx;
                __stcg(&A->q_last, qt);
                __stcg(&A->q_sum, __ldcg(&A->q_sum) + qt);
                __stcg(&A->q_sum2, __ldcg(&A->q_sum2) + qt * qt);
                __stcg(&A->q_n, __ldcg(&A->q_n) + 1.0);
                atomicExch(&A->count, 0u);
            }
        }
    }
}
#undef LB_SMP
#undef LB_SMC

// The single-domain step at 64 and 128 threads gives the compiler only its
// block size (151 registers: 12 warps per SM, 6 blocks of 64 or 3 of 128).
// This measured 5 % faster on 4096^2 and 8 % on 8192^2 than the same
// occupancy requested through __launch_bounds__' minimum blocks (148
// registers, a different schedule), and faster than register caps of 144
// (4 %) or 136 (6 %). 256 threads keep 2 blocks per SM through the
// minimum-blocks bound (lb_step_dual_lb: 118 registers).
template <int BD, int MINB, class T>
__global__ void __launch_bounds__(BD) lb_step_dual(const StepParams P) {
    step_body<BD, T>(P, P, blockIdx.x);
}

template <int BD, int MINB, class T>
__global__ void __launch_bounds__(BD, MINB) lb_step_dual_lb(const StepParams P) {
    step_body<BD, T>(P, P, blockIdx.x);
}

// the step kernel of a block size
template <int BD, int MINB, class T>
constexpr auto dual_kernel() {
    if constexpr (BD == 256) return lb_step_dual_lb<BD, MINB, T>;
    else return lb_step_dual<BD, MINB, T>;
}

// The forward intermediates of one step for the adjoint (paired FP32); with
// OUT also the step itself (f_out, th_out), with QF also q(t).
template <int BD, int MINB, bool OUT, bool QF>
__global__ void __launch_bounds__(BD, MINB) lb_step_recompute(const StepParams P, const __grid_constant__ RecomputeOut R) {
    step_body<BD, P2, true, false, OUT, QF>(P, P, blockIdx.x, &R);
}

// Many independent simulations in one launch (the boiling-curve batch): the
// blocks of instance i are [block_off[i], block_off[i+1]); each block copies
// its instance's parameter record to shared memory (sP) and returns the
// block's index within its instance.
template <int BD>
__device__ __forceinline__ int batch_instance(const StepParams* __restrict__ table, const int* __restrict__ block_off,
                                              int n, StepParams& sP) {
    __shared__ int s_inst;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n - 1;  // largest i with block_off[i] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (block_off[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_inst = lo;
    }
    __syncthreads();
    const int inst = s_inst;
    constexpr int NW = (int)(sizeof(StepParams) / sizeof(int));
    static_assert(sizeof(StepParams) % sizeof(int) == 0, "StepParams is copied as ints");
    for (int k = threadIdx.x; k < NW; k += BD)
        reinterpret_cast<int*>(&sP)[k] = __ldg(reinterpret_cast<const int*>(table + inst) + k);
    __syncthreads();
    return (int)blockIdx.x - block_off[inst];
}

// The batch with every model constant from the instance's record.
template <int BD, int MINB, class T>
__global__ void __launch_bounds__(BD, MINB) lb_step_batch(const StepParams* __restrict__ table,
                                                        const int* __restrict__ block_off, int n) {
    __shared__ StepParams sP;
    const int b = batch_instance<BD>(table, block_off, n, sP);
    step_body<BD, T>(sP, sP, b);
}

// The batch with the model constants shared by all instances (K, in the
// parameter bank); the table supplies each instance's buffers, sizes,
// launch shape, wettability and rho_ave.
template <int BD, int MINB, class T>
__global__ void __launch_bounds__(BD, MINB) lb_step_batch_k(const StepParams K, const StepParams* __restrict__ table,
                                                          const int* __restrict__ block_off, int n) {
    __shared__ StepParams sP;
    const int b = batch_instance<BD>(table, block_off, n, sP);
    step_body<BD, T>(sP, K, b);
}

// ---------------------------------------------------------------------------
// The persistent batch: one launch advances every instance by `nsteps` steps.
//
// The instances' tiles (a pair of column strips x a segment of rows, the
// unit one block of the per-step kernel computes) are dealt out to a fixed,
// co-resident grid (a cooperative launch); block g takes tiles
// tile_off[g] .. tile_off[g+1]-1 in that order, step after step. A tile may
// start step k once every tile of its instance has finished step k-1:
// its pulled rows and the strips beside it are then complete (read after
// write), and no tile of the instance still reads the buffer step k writes
// (write after read). arrive[i] counts the tiles of instance i that have
// finished a step since the launch began (zeroed before each launch), so
// the wait is arrive[i] >= k * ntiles[i]. The wait spins at most
// `wait_limit` polls (with a short sleep between them); a block that gives
// up sets ERR_TIMEOUT in its instance's fault flags and leaves the kernel,
// which lets every block waiting on it give up in turn, so the launch always
// ends. The step's input state is read with plain loads, which after the
// acquiring wait and the barrier see the other SMs' writes (the read-only
// path could serve copies cached before them), and every tile runs the same
// step body as the per-step kernel, so results are bit-identical to it.
// ---------------------------------------------------------------------------

// Poll *p until it reaches `target`, at most `limit` times; true if reached.
__device__ __forceinline__ bool wait_at_least(const unsigned* p, unsigned target, unsigned long long limit) {
    for (unsigned long long it = 0;; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return true;
        if (it >= limit) return false;
        __nanosleep(64);
    }
}

// The most tiles one block of the persistent batch schedules by readiness
// (more than this many are taken in order).
constexpr int PERSIST_MAX_TILES = 64;

template <int BD, int MINB, bool SK>
__global__ void __launch_bounds__(BD, MINB) lb_batch_persist(const StepParams K, const PersistArgs A) {
    __shared__ StepParams sP;
    __shared__ int s_next[PERSIST_MAX_TILES];  // next step of each of the block's tiles
    __shared__ int s_pick;
    const int t0 = A.tile_off[blockIdx.x], t1 = A.tile_off[blockIdx.x + 1];
    const int m = t1 - t0;
    const bool by_ready = m <= PERSIST_MAX_TILES;
    for (int j = threadIdx.x; j < PERSIST_MAX_TILES; j += BD) s_next[j] = 0;
    __syncthreads();
    // whether tile j may run its next step: every tile of its instance has
    // finished the previous one
    auto ready = [&](int j, int k) {
        const int inst = A.tiles[t0 + j].x;
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(A.arrive + inst) : "memory");
        return k == 0 || v >= (unsigned)k * (unsigned)A.ntiles[inst];
    };
    int last = m - 1, done_in_order = 0;
    for (;;) {
        // thread 0 picks the next tile: with few tiles per block the first
        // ready one after the last tile run (round robin), so a block never
        // idles while one of its tiles can go on; otherwise the tiles in
        // order, step after step. -2: all done; -3: a wait ran out.
        if (threadIdx.x == 0) {
            int pick = -2;
            if (by_ready) {
                unsigned long long polls = 0;
                for (;;) {
                    bool left = false;
                    pick = -1;
                    for (int d = 1; d <= m; ++d) {
                        const int j = (last + d) % m;
                        if (s_next[j] >= A.nsteps) continue;
                        left = true;
                        if (ready(j, s_next[j])) {
                            pick = j;
                            break;
                        }
                    }
                    if (!left) {
                        pick = -2;
                        break;
                    }
                    if (pick >= 0) break;
                    if (polls++ >= A.wait_limit) {
                        pick = -3;
                        break;
                    }
                    __nanosleep(64);
                }
            } else if (done_in_order < m * A.nsteps) {
                const int j = done_in_order % m, k = done_in_order / m;
                pick = wait_at_least(A.arrive + A.tiles[t0 + j].x, (unsigned)k * (unsigned)A.ntiles[A.tiles[t0 + j].x],
                                     k == 0 ? 0ull : A.wait_limit) || k == 0 ? j : -3;
                if (pick >= 0) s_next[0] = k;  // the step to run
            }
            if (pick == -3) {  // latch the timeout on an unfinished tile's instance
                for (int j = 0; j < m; ++j)
                    if (!by_ready || s_next[j] < A.nsteps) {
                        atomicOr(&A.table[A.tiles[t0 + j].x].acc->err, ERR_TIMEOUT);
                        break;
                    }
            }
            s_pick = pick;
        }
        __syncthreads();
        const int pick = s_pick;
        if (pick < 0) return;  // all done, or given up
        const int k = by_ready ? s_next[pick] : s_next[0];
        const int2 tl = A.tiles[t0 + pick];
        const StepParams* src = A.table + (k & 1) * A.n + tl.x;
        constexpr int NW = (int)(sizeof(StepParams) / sizeof(int));
        for (int w = threadIdx.x; w < NW; w += BD)
            reinterpret_cast<int*>(&sP)[w] = __ldg(reinterpret_cast<const int*>(src) + w);
        __syncthreads();
        step_body<BD, P2, false, true>(sP, SK ? K : sP, tl.y);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(A.arrive + tl.x, 1u);
            if (by_ready) ++s_next[pick];
            else ++done_in_order;
            last = pick;
        }
        __syncthreads();
    }
}

namespace {

// blocks per SM the batch kernels (per-step and persistent) are compiled for:
// at 64 threads the single-domain step's 6 (up to 168 registers, and shared
// memory left to L1 for the pulled rows) measured faster than 8 (128
// registers) on the 48-instance curve batch: 0.177 against 0.185 ms per
// batched step, both launch forms
constexpr int BATCH_MINB64 = 6, BATCH_MINB128 = 4;

template <int BD, int MINB, class T>
struct DualKernel {
    static size_t smem() { return sizeof(float2) * ((size_t)SM_ROWS * (BD + 2) + 4 * RING * BD); }
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(dual_kernel<BD, MINB, T>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem());
    }
    static cudaError_t occupancy(int* n) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, dual_kernel<BD, MINB, T>(), BD, smem());
    }
    static cudaError_t launch(const StepParams& P, int nblocks, cudaStream_t st) {
        dual_kernel<BD, MINB, T>()<<<nblocks, BD, smem(), st>>>(P);
        return cudaGetLastError();
    }
    static cudaError_t prepare_batch() {
        return cudaFuncSetAttribute(lb_step_batch<BD, MINB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem());
    }
    static cudaError_t occupancy_batch(int* n) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lb_step_batch<BD, MINB, T>, BD, smem());
    }
    static cudaError_t occupancy_batch_k(int* n) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lb_step_batch_k<BD, MINB, T>, BD, smem());
    }
    static cudaError_t launch_batch(const StepParams* table, const int* off, int n, int nblocks, cudaStream_t st) {
        lb_step_batch<BD, MINB, T><<<nblocks, BD, smem(), st>>>(table, off, n);
        return cudaGetLastError();
    }
    static cudaError_t prepare_batch_k() {
        return cudaFuncSetAttribute(lb_step_batch_k<BD, MINB, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem());
    }
    static cudaError_t launch_batch_k(const StepParams& K, const StepParams* table, const int* off, int n,
                                      int nblocks, cudaStream_t st) {
        lb_step_batch_k<BD, MINB, T><<<nblocks, BD, smem(), st>>>(K, table, off, n);
        return cudaGetLastError();
    }
    template <bool SK>
    static cudaError_t prepare_persist() {
        return cudaFuncSetAttribute(lb_batch_persist<BD, MINB, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem());
    }
    template <bool SK>
    static cudaError_t occupancy_persist(int* n) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lb_batch_persist<BD, MINB, SK>, BD, smem());
    }
    // a cooperative launch: the runtime refuses it unless every block can be
    // resident at once, which the blocks' waits on one another need
    template <bool SK>
    static cudaError_t launch_persist(const StepParams& K, const PersistArgs& A, int nblocks, cudaStream_t st) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nblocks);
        cfg.blockDim = dim3(BD);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, lb_batch_persist<BD, MINB, SK>, K, A);
    }
};

// the instantiations a launch can pick: (block size, paired FP32 or scalar).
// The single-domain step runs 12 warps per SM (6 blocks of 64 or 3 of 128
// with ~151 registers a thread), not 16 (8 x 64 or 4 x 128 at 128
// registers): within 128 registers the compiler spends ~50 more instructions
// per cell on copies and recomputation, which costs more than the four warps
// gain. For the single-domain kernels at 64 and 128 threads MINB names the
// intended blocks per SM only (the occupancy query sizes the grid;
// lb_step_dual gives the compiler its block size alone). The
// batched step keeps 128 registers: with its parameters in shared memory it
// ran 7 % slower with the larger budget.
cudaError_t dual_prepare_t() {
    cudaError_t e = DualKernel<64, 6, P2>::prepare();
    if (e == cudaSuccess) e = DualKernel<128, 3, P2>::prepare();
    if (e == cudaSuccess) e = DualKernel<256, 2, P2>::prepare();
    return e;
}

cudaError_t batch_prepare_t() {
    cudaError_t e = DualKernel<64, BATCH_MINB64, P2>::prepare_batch();
    if (e == cudaSuccess) e = DualKernel<128, BATCH_MINB128, P2>::prepare_batch();
    if (e == cudaSuccess) e = DualKernel<64, BATCH_MINB64, P2>::prepare_batch_k();
    if (e == cudaSuccess) e = DualKernel<128, BATCH_MINB128, P2>::prepare_batch_k();
    if (e == cudaSuccess) e = DualKernel<64, BATCH_MINB64, P2>::prepare_persist<true>();
    if (e == cudaSuccess) e = DualKernel<64, BATCH_MINB64, P2>::prepare_persist<false>();
    if (e == cudaSuccess) e = DualKernel<128, BATCH_MINB128, P2>::prepare_persist<true>();
    if (e == cudaSuccess) e = DualKernel<128, BATCH_MINB128, P2>::prepare_persist<false>();
    return e;
}

cudaError_t dual_occupancy_t(int block_x, int* n) {
    if (block_x == 64) return DualKernel<64, 6, P2>::occupancy(n);
    if (block_x == 128) return DualKernel<128, 3, P2>::occupancy(n);
    return DualKernel<256, 2, P2>::occupancy(n);
}

cudaError_t dual_launch_t(const StepParams& P, const Launch& L, cudaStream_t st) {
    const int nb = L.nstrips * L.nseg;
    if (L.block_x == 64) return DualKernel<64, 6, P2>::launch(P, nb, st);
    if (L.block_x == 128) return DualKernel<128, 3, P2>::launch(P, nb, st);
    return DualKernel<256, 2, P2>::launch(P, nb, st);
}

}  // namespace

bool dual_supported(int block_x) { return block_x == 64 || block_x == 128 || block_x == 256; }

namespace {

template <int BD, int MINB>
cudaError_t recompute_prepare_t() {
    const int sm = (int)DualKernel<BD, MINB, P2>::smem();
    cudaError_t e = cudaFuncSetAttribute(lb_step_recompute<BD, MINB, false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lb_step_recompute<BD, MINB, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lb_step_recompute<BD, MINB, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

template <int BD, int MINB>
cudaError_t recompute_t(const StepParams& P, const RecomputeOut& R, bool out, bool heat, int nblocks,
                        cudaStream_t st) {
    const size_t sm = DualKernel<BD, MINB, P2>::smem();
    if (out && heat) lb_step_recompute<BD, MINB, true, true><<<nblocks, BD, sm, st>>>(P, R);
    else if (out) lb_step_recompute<BD, MINB, true, false><<<nblocks, BD, sm, st>>>(P, R);
    else lb_step_recompute<BD, MINB, false, false><<<nblocks, BD, sm, st>>>(P, R);
    return cudaGetLastError();
}

}  // namespace

cudaError_t dual_recompute(const StepParams& P, const RecomputeOut& R, bool out, bool heat, const Launch& L,
                           cudaStream_t st) {
    if (heat && !out) return cudaErrorInvalidValue;
    const int nb = L.nstrips * L.nseg;
    if (L.block_x == 64) return recompute_t<64, 6>(P, R, out, heat, nb, st);
    if (L.block_x == 128) return recompute_t<128, 3>(P, R, out, heat, nb, st);
    if (L.block_x == 256) return recompute_t<256, 2>(P, R, out, heat, nb, st);
    return cudaErrorInvalidValue;
}

cudaError_t dual_prepare() {
    cudaError_t e = dual_prepare_t();
    if (e == cudaSuccess) e = recompute_prepare_t<64, 6>();
    if (e == cudaSuccess) e = recompute_prepare_t<128, 3>();
    if (e == cudaSuccess) e = recompute_prepare_t<256, 2>();
    return e;
}

cudaError_t dual_occupancy(int block_x, int* n) { return dual_occupancy_t(block_x, n); }

cudaError_t launch_step(const StepParams& P, const Launch& L, cudaStream_t st) { return dual_launch_t(P, L, st); }

bool batch_supported(int block_x) { return block_x == 64 || block_x == 128; }

cudaError_t batch_prepare() { return batch_prepare_t(); }

cudaError_t batch_occupancy(int block_x, bool shared_k, int* n) {
    if (shared_k)
        return block_x == 64 ? DualKernel<64, BATCH_MINB64, P2>::occupancy_batch_k(n)
                             : DualKernel<128, BATCH_MINB128, P2>::occupancy_batch_k(n);
    return block_x == 64 ? DualKernel<64, BATCH_MINB64, P2>::occupancy_batch(n) : DualKernel<128, BATCH_MINB128, P2>::occupancy_batch(n);
}

cudaError_t persist_occupancy(int block_x, bool shared_k, int* n) {
    if (block_x == 64)
        return shared_k ? DualKernel<64, BATCH_MINB64, P2>::occupancy_persist<true>(n) : DualKernel<64, BATCH_MINB64, P2>::occupancy_persist<false>(n);
    return shared_k ? DualKernel<128, BATCH_MINB128, P2>::occupancy_persist<true>(n) : DualKernel<128, BATCH_MINB128, P2>::occupancy_persist<false>(n);
}

cudaError_t persist_launch(int block_x, const StepParams* K, const PersistArgs& A, int nblocks, cudaStream_t st) {
    const StepParams k0 = K ? *K : StepParams{};
    if (block_x == 64)
        return K ? DualKernel<64, BATCH_MINB64, P2>::launch_persist<true>(k0, A, nblocks, st)
                 : DualKernel<64, BATCH_MINB64, P2>::launch_persist<false>(k0, A, nblocks, st);
    return K ? DualKernel<128, BATCH_MINB128, P2>::launch_persist<true>(k0, A, nblocks, st)
             : DualKernel<128, BATCH_MINB128, P2>::launch_persist<false>(k0, A, nblocks, st);
}

cudaError_t batch_launch(int block_x, const StepParams* table, const int* block_off, int n, int nblocks,
                         const StepParams* K, cudaStream_t st) {
    if (K)
        return block_x == 64 ? DualKernel<64, BATCH_MINB64, P2>::launch_batch_k(*K, table, block_off, n, nblocks, st)
                             : DualKernel<128, BATCH_MINB128, P2>::launch_batch_k(*K, table, block_off, n, nblocks, st);
    return block_x == 64 ? DualKernel<64, BATCH_MINB64, P2>::launch_batch(table, block_off, n, nblocks, st)
                         : DualKernel<128, BATCH_MINB128, P2>::launch_batch(table, block_off, n, nblocks, st);
}

}  // namespace lbgpu
