// Off-hot-path kernels: initial state, macroscopic fields, FP64 mass sum,
// and the pressure probe run after a step when probes are set (Fig. 3).
#include "lb_internal.h"

namespace lbgpu {

namespace {

__constant__ float kW[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                            1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};

// The per-cell kernels below take rows blockIdx.y, blockIdx.y + gridDim.y, ...
// (gridDim.y is capped at the 65535 limit of the launch).
__global__ void init_kernel(const StepParams P, const float* __restrict__ rho0, float* f, float* th) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.Lx) return;
    for (int y = blockIdx.y; y < P.Ly; y += gridDim.y) {
        const int i = y * P.pitch + x;
        const float r = rho0[i];
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a * P.plane + i] = kW[a] * r;
        float t = 0.f;
        if (P.bc != BC_PERIODIC && y == 0) t = P.thb[x];
        th[i] = t;
    }
}

// Pass 1 at one cell: the pulled populations give rho, psi and the momentum
// sums.
__device__ __forceinline__ void macro1_cell(const StepParams& P, float* scr, int x, int y) {
    const int xm = x == 0 ? P.Lx - 1 : x - 1;
    const int xp = x == P.Lx - 1 ? 0 : x + 1;
    float f[9], th;
    load_row(P, y, x, xm, xp, f, th);
    wall_fill(P, y, f);
    float rho = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) rho += f[a];
    const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const float jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    bool bad = false;
    const float psi = eos_psi(rho, P.Ts + th, P, bad);
    if (bad) atomicOr(&P.acc->err, ERR_EOS);
    const int i = y * P.pitch + x;
    scr[i] = rho;
    scr[P.plane + i] = psi;
    scr[2 * P.plane + i] = jx;
    scr[3 * P.plane + i] = jy;
}

// Pass 2 at one cell.
__device__ __forceinline__ void macro2_cell(const StepParams& P, const float* __restrict__ scr, float* orho,
                                            float* oux, float* ouy, float* oT, int ostride, int x, int y) {
    const int Lx = P.Lx, Ly = P.Ly, pitch = P.pitch;
    const bool periodic = P.bc == BC_PERIODIC;
    const bool wall = !periodic && (y == 0 || y == Ly - 1);
    const float* psi = scr + P.plane;
    const int i = y * pitch + x;
    const float rho = scr[i], ps = psi[i];
    float Fmx = 0.f, Fmy = 0.f;
    if (!wall || P.ghost) {
        const int ym = periodic ? wrap(y - 1, Ly) : (y == 0 ? 0 : y - 1);
        const int yp = periodic ? wrap(y + 1, Ly) : (y == Ly - 1 ? Ly - 1 : y + 1);
        const int xm = x == 0 ? Lx - 1 : x - 1, xp = x == Lx - 1 ? 0 : x + 1;
        float pm[3] = {psi[ym * pitch + xm], psi[ym * pitch + x], psi[ym * pitch + xp]};
        float pc[3] = {psi[y * pitch + xm], ps, psi[y * pitch + xp]};
        float pn[3] = {psi[yp * pitch + xm], psi[yp * pitch + x], psi[yp * pitch + xp]};
        float sx, sy;
        psi_sum(pm + 1, pc + 1, pn + 1, sx, sy);
        Fmx = -P.G * ps * sx;
        Fmy = -P.G * ps * sy;
    }
    float Fx = Fmx, Fy = Fmy;
    if (!wall) {
        if (!periodic && y == 1) Fy += P.gw6 * ps * ps;
        Fy -= P.g * (rho - P.rho_ave);
    }
    const int o = y * ostride + x;
    if (orho) orho[o] = rho;
    if (oux) oux[o] = (scr[2 * P.plane + i] + 0.5f * Fx) / rho;
    if (ouy) ouy[o] = (scr[3 * P.plane + i] + 0.5f * Fy) / rho;
    if (oT) oT[o] = P.Ts + P.th_in[i];
}

// Pass 1: pulled populations -> rho, psi, momentum sums into scratch planes.
__global__ void macro_pass1(const StepParams P, float* scr) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.Lx) return;
    for (int y = blockIdx.y; y < P.Ly; y += gridDim.y) macro1_cell(P, scr, x, y);
}

// Pass 2: forces (Eqs. 7, 9, 22) and u = (j + F/2)/rho (Eq. 6).
__global__ void macro_pass2(const StepParams P, const float* __restrict__ scr, float* orho, float* oux,
                            float* ouy, float* oT, int ostride) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= P.Lx) return;
    for (int y = blockIdx.y; y < P.Ly; y += gridDim.y) macro2_cell(P, scr, orho, oux, ouy, oT, ostride, x, y);
}

__global__ void mass_kernel(const StepParams P, const float* __restrict__ f) {
    __shared__ double red[32];
    double s = 0.0;
    const long long n = 9LL * P.Ly * P.Lx;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long a = k / ((long long)P.Ly * P.Lx);
        const long long rem = k - a * P.Ly * P.Lx;
        const int y = (int)(rem / P.Lx), x = (int)(rem - (long long)y * P.Lx);
        s += (double)f[a * P.plane + (long long)y * P.pitch + x];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(&P.acc->mass, t);
    }
}

}  // namespace

cudaError_t launch_init(const StepParams& P, const float* rho0, float* f, float* th, cudaStream_t st) {
    dim3 grid((P.Lx + 127) / 128, P.Ly < 65535 ? P.Ly : 65535);
    init_kernel<<<grid, 128, 0, st>>>(P, rho0, f, th);
    return cudaGetLastError();
}

cudaError_t launch_macro(const StepParams& P, float* scratch, float* rho, float* ux, float* uy, float* T,
                         int ostride, cudaStream_t st) {
    dim3 grid((P.Lx + 127) / 128, P.Ly < 65535 ? P.Ly : 65535);
    macro_pass1<<<grid, 128, 0, st>>>(P, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    macro_pass2<<<grid, 128, 0, st>>>(P, scratch, rho, ux, uy, T, ostride);
    return cudaGetLastError();
}

cudaError_t launch_mass(const StepParams& P, const float* f, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&P.acc->mass, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    mass_kernel<<<256, 256, 0, st>>>(P, f);
    return cudaGetLastError();
}

// One block: thread k < n handles probe k. rho^t is the sum of the stored
// post-collision populations (the collision conserves it), T^t = T_s +
// theta^t, and p the Peng-Robinson pressure of Eq. 21 in FP64.
__global__ void probe_kernel(const ProbeArgs A) {
    const int k = threadIdx.x;
    unsigned long long* count = reinterpret_cast<unsigned long long*>(A.ring);
    const unsigned long long s = *count;
    __syncthreads();
    if (k < A.n) {
        const int i = A.y[k] * A.pitch + A.x[k];
        float rho = 0.f;
#pragma unroll
        for (int a = 0; a < 9; ++a) rho += A.f[a * A.plane + i];
        const double r = rho, T = A.Ts + (double)A.th[i];
        const double br = A.b * r, ph = A.k0 - A.k1 * sqrt(T);
        const double p = A.R * r * T / (1.0 - br) - A.a * ph * ph * r * r / (1.0 + 2.0 * br - br * br);
        float* rec = A.ring + 64 + 4 * ((size_t)k * A.cap + (size_t)(s % (unsigned long long)A.cap));
        rec[0] = rho;
        rec[1] = (float)T;
        rec[2] = (float)p;
        rec[3] = 0.f;
    }
    __syncthreads();
    if (k == 0) *count = s + 1;
}

cudaError_t launch_probe(const ProbeArgs& A, cudaStream_t st) {
    probe_kernel<<<1, 32, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace lbgpu
