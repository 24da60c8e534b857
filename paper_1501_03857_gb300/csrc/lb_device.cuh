// Device-side definitions shared by the kernels of the GB300 boiling step.
//
// Lattice: D2Q9 with e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1)
// e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1) (Sec. 2). Fields are pitched
// row-major [y][pitch] FP32, populations are 9 such planes (SoA).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbgpu {

constexpr int HALO = 5;    // x-halo columns per side recomputed by a block
// the narrowest block (64 threads) covers 2 (64 - 2 HALO) = 108 columns, so a
// grid has at most ceil(Lx / 108) strips: the heat-flux slots per instance
constexpr int MIN_STRIP_COLS = 2 * (64 - 2 * HALO);
constexpr int RING = 4;    // rows kept per stencil field in shared memory
constexpr int TRING = 8;   // rows kept of theta^t
constexpr int SM_ROWS = 7 * RING + TRING;  // psi rho vx vy u2 u3 u4 + theta

enum { BC_WALLS = 0, BC_TOP_OUTFLOW = 1, BC_PERIODIC = 2 };
enum : unsigned { ERR_EOS = 1u, ERR_NONFINITE = 2u, ERR_BOUNDS = 4u, ERR_TIMEOUT = 8u };

// FP64 device accumulators (wall heat flux of Sec. 3.2, mass, fault flags).
struct Acc {
    double spare;
    double q_last;      // q(t) of the last completed step
    double q_sum, q_sum2, q_n;
    double mass;
    unsigned int count; // bottom blocks that added their partial this step
    unsigned int err;   // ERR_* bits
    double pad[2];
};

// Everything one launch of the step needs, passed by value.
struct StepParams {
    const float* f_in;
    float* f_out;
    const float* th_in;
    float* th_out;
    const float* thb;   // theta_b(x) = T_b(x) - T_s on the bottom wall
    Acc* acc;
    // one slot per column strip of the bottom segment: the strip's sum of
    // q_w for the step in flight, folded in strip order by the last strip
    double* qpart;
    int Lx, Ly, pitch, plane;
    int bc, ghost, isothermal;
    int nout, nstrips, seg_h;
    // Peng-Robinson EOS (Eq. 21): phi(T) = (k0 - k1 sqrt(T))^2 with
    // k0 = 1 + kappa, k1 = kappa / sqrt(Tc); psi^2 = two_over_G (p - rho/3).
    float Ts, a, b, R, two_over_G, k0, k1, G;
    float k0k1, k1k1;  // phi'(T) = k1^2 - k0 k1 / sqrt(T)
    // MRT collision (Eqs. 2, 4, 8)
    float s_e, s_z, s_q, sig_e, sig_z;
    float rho_v, inv_drho, tau_v, dtau;
    // forces (Eqs. 9, 22); gw6 = G_w/6 is -G_w sum_a omega_a s e_a,y on row 1
    float g, rho_ave, gw6;
    // temperature (Eq. 18): chi = c_v chi / c_v, cvchi = c_v chi
    float chi, cvchi, inv_cv;
    // the constants of the paired FP32 arithmetic, each duplicated into a
    // float2 so that a paired instruction can take it from the parameter
    // bank as it is (set_pairs)
    float2 kp[27];
};

enum {
    KP_TS, KP_K1N, KP_K0, KP_B, KP_R, KP_A, KP_2G, KP_K0K1N, KP_K1K1, KP_CHI6,
    KP_SE36N, KP_KE6, KP_KESIG, KP_SZ12N, KP_KZ6N, KP_KZSIGN, KP_SQ6, KP_SQ12N, KP_DTAU4, KP_TAUV4,
    KP_GN12, KP_GW6, KP_GN, KP_RHOAVE, KP_CHI144, KP_RCV12, KP_ACV12, KP_COUNT
};

// Fill kp from the scalar fields (after any of them changes).
inline void set_pairs(StepParams& P) {
    static_assert(KP_COUNT == sizeof(P.kp) / sizeof(P.kp[0]), "kp size");
    const float G2 = P.G * P.G * (1.f / 144.f);
    const float ke = (1.f - 0.5f * P.s_e) * (1.f / 36.f), kz = (1.f - 0.5f * P.s_z) * (1.f / 36.f);
    const float v[KP_COUNT] = {P.Ts, -P.k1, P.k0, P.b, P.R, P.a, P.two_over_G, -P.k0k1, P.k1k1, P.chi * (1.f / 6.f),
                               -P.s_e * (1.f / 36.f), 6.f * ke, ke * P.sig_e * G2, -P.s_z * (1.f / 12.f), -6.f * kz,
                               -kz * P.sig_z * G2, P.s_q * (1.f / 6.f), -P.s_q * (1.f / 12.f), 4.f * P.dtau,
                               4.f * P.tau_v, -P.G * (1.f / 12.f), P.gw6, -P.g, P.rho_ave, P.chi * (1.f / 144.f),
                               P.R * P.inv_cv * (1.f / 12.f), P.a * P.inv_cv * (1.f / 12.f)};
    for (int i = 0; i < KP_COUNT; ++i) P.kp[i] = make_float2(v[i], v[i]);
}

__device__ __forceinline__ int wrap(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ bool finite_f(float v) { return fabsf(v) <= 3.402823466e38f; }

// Checked build (-DLB_CHECKED, liblbboil_checked.so): every global and
// shared-memory access of the fused step goes through these; an address
// outside its buffer sets ERR_BOUNDS and the access is skipped (a load reads
// 0) instead of faulting. In the normal build they are the plain accesses.
#ifdef LB_CHECKED
__device__ __forceinline__ bool lb_inside(const void* p, const void* base, size_t bytes, size_t width, Acc* acc) {
    const char* c = static_cast<const char*>(p);
    const char* b = static_cast<const char*>(base);
    if (base != nullptr && c >= b && c + width <= b + bytes) return true;
    atomicOr(&acc->err, ERR_BOUNDS);
    return false;
}
__device__ __forceinline__ float lb_ldg(const float* p, const float* base, size_t n, Acc* acc) {
    return lb_inside(p, base, n * sizeof(float), sizeof(float), acc) ? __ldg(p) : 0.f;
}
__device__ __forceinline__ void lb_st(float* p, float v, const float* base, size_t n, Acc* acc) {
    if (lb_inside(p, base, n * sizeof(float), sizeof(float), acc)) *p = v;
}
__device__ __forceinline__ float lb_ldco(const float* p, const float* base, size_t n, Acc* acc) {
    return lb_inside(p, base, n * sizeof(float), sizeof(float), acc) ? *p : 0.f;
}
#else
__device__ __forceinline__ float lb_ldg(const float* p, const float*, size_t, Acc*) { return __ldg(p); }
__device__ __forceinline__ float lb_ldco(const float* p, const float*, size_t, Acc*) { return *p; }
__device__ __forceinline__ void lb_st(float* p, float v, const float*, size_t, Acc*) { *p = v; }
#endif
// Loads of the step's input state: through the read-only path in a kernel
// that runs one step (lb_ldg), as plain coherent loads (lb_ldco) in the
// persistent batch, where other blocks rewrite the buffers during the launch:
// the read-only path may serve data it cached before that; a plain load after
// the block's acquire of the other blocks' progress sees their writes.
template <bool CO>
__device__ __forceinline__ float lb_ld(const float* p, const float* base, size_t n, Acc* acc) {
    if constexpr (CO) return lb_ldco(p, base, n, acc);
    else return lb_ldg(p, base, n, acc);
}

// psi(rho, T) = sqrt(2 (p_EOS - rho c_s^2) / G), c = 1 (Sec. 2 and Eq. 21).
__device__ __forceinline__ float eos_psi(float rho, float T, const StepParams& P, bool& bad) {
    const float sT = sqrtf(T);
    float ph = P.k0 - P.k1 * sT;
    ph *= ph;
    const float br = P.b * rho;
    const float p = rho * P.R * T / (1.f - br) - P.a * ph * rho * rho / (1.f + 2.f * br - br * br);
    float arg = P.two_over_G * (p - rho * (1.f / 3.f));
    if (arg < 0.f) {
        bad = true;
        arg = 0.f;
    }
    return sqrtf(arg);
}

// Pulled populations of row y at column x (Eq. 3: f_a(x) = f*_a(x - e_a)).
// Populations whose source lies outside a wall are left 0 and filled by
// Zou-He; with the outflow top the source row is clamped to the top row.
__device__ __forceinline__ void load_row(const StepParams& P, int y, int x, int xm, int xp,
                                         float (&f)[9], float& th) {
    const float* __restrict__ F = P.f_in;
    const int pl = P.plane, pitch = P.pitch;
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
    const int rc = y * pitch, rm = ym * pitch, rp = yp * pitch;
    f[0] = __ldg(F + 0 * pl + rc + x);
    f[1] = __ldg(F + 1 * pl + rc + xm);
    f[3] = __ldg(F + 3 * pl + rc + xp);
    f[2] = okm ? __ldg(F + 2 * pl + rm + x) : 0.f;
    f[5] = okm ? __ldg(F + 5 * pl + rm + xm) : 0.f;
    f[6] = okm ? __ldg(F + 6 * pl + rm + xp) : 0.f;
    f[4] = okp ? __ldg(F + 4 * pl + rp + x) : 0.f;
    f[7] = okp ? __ldg(F + 7 * pl + rp + xp) : 0.f;
    f[8] = okp ? __ldg(F + 8 * pl + rp + xm) : 0.f;
    th = __ldg(P.th_in + rc + x);
}

// Zou-He no-slip (u = 0) fill of the unknown populations on the wall rows
// (Sec. 3.1): zero momentum and bounce-back of the normal non-equilibrium
// part. Bottom unknowns 2, 5, 6; top unknowns 4, 7, 8 (walls only).
__device__ __forceinline__ void wall_fill(const StepParams& P, int y, float (&f)[9]) {
    if (P.bc != BC_PERIODIC && y == 0) {
        const float d = 0.5f * (f[1] - f[3]);
        f[2] = f[4];
        f[5] = f[7] - d;
        f[6] = f[8] + d;
    }
    if (P.bc == BC_WALLS && y == P.Ly - 1) {
        const float d = 0.5f * (f[1] - f[3]);
        f[4] = f[2];
        f[7] = f[5] + d;
        f[8] = f[6] - d;
    }
}

// sum_a w_a psi(x + e_a) e_a with w = 1/3 (axis), 1/12 (diagonal), Eq. 7;
// pm, pc, pn point at column x of rows y-1, y, y+1.
__device__ __forceinline__ void psi_sum(const float* pm, const float* pc, const float* pn,
                                        float& sx, float& sy) {
    sx = (pc[1] - pc[-1]) * (1.f / 3.f) + ((pn[1] - pm[-1]) + (pm[1] - pn[-1])) * (1.f / 12.f);
    sy = (pn[0] - pm[0]) * (1.f / 3.f) + ((pn[1] - pm[-1]) + (pn[-1] - pm[1])) * (1.f / 12.f);
}

}  // namespace lbgpu
