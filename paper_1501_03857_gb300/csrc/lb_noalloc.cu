// lb_fields_noalloc: the macroscopic-field computation of lb_fields for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or allocator hook, a host process restricted from
// creating allocations after start-up, or a real-time loop that must not
// touch the allocator. lb_fields itself needs no allocation either, but only
// because lb_init received a caller-allocated workspace; this entry point
// needs no handle and no workspace. Its scratch (four planes: density,
// pseudopotential and the two momentum sums of the pulled populations, plus
// the fault-flag word) lives in the file-scope array below. With the CUDA
// runtime's lazy module loading (its default) the array is placed in device
// memory when the first call on a device looks up its address, and that
// device keeps it until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "lb.h"
#include "lb_internal.h"

using namespace lbgpu;

namespace {

// Scratch: one Acc record (fault flags) in the first 256 bytes, then four
// planes of LB_NOALLOC_MAX_CELLS floats.
constexpr size_t kAccBytes = 256;
constexpr size_t kScratchBytes = kAccBytes + 4 * sizeof(float) * (size_t)LB_NOALLOC_MAX_CELLS;
static_assert(sizeof(Acc) <= kAccBytes, "Acc must fit its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// The symbol's device address for the current device, looked up once per
// device (the name g_noalloc_scratch is only a host-side stand-in in host
// code and must never be passed to a kernel itself).
cudaError_t scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

int fail(int code, const char* msg) {
    set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int lb_fields_noalloc(const lb_grid* grid, const lb_eos* eos, const lb_thermal* th, double Gw,
                                 double rho_ave, const float* fpost, const float* theta, float* rho, float* ux,
                                 float* uy, float* T, void* stream) {
    if (!grid || !eos || !th || !fpost || !theta) return fail(LB_E_INVAL, "null argument");
    if (grid->Lx < 1 || grid->Ly < 3 || grid->bc_y < LB_BC_WALLS || grid->bc_y > LB_BC_PERIODIC)
        return fail(LB_E_INVAL, "bad grid (need Lx >= 1, Ly >= 3, bc_y in 0..2)");
    // the call waits for the stream before it returns, which a stream under
    // capture does not allow: refuse before anything is enqueued, so that the
    // caller's capture stays valid
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(st, &cap);
    if (ce != cudaSuccess) return fail(LB_E_CUDA, cudaGetErrorString(ce));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(LB_E_INVAL, "the stream is being captured; lb_fields_noalloc synchronises its stream");
    const long long cells = (long long)grid->Lx * grid->Ly;
    if (cells > LB_NOALLOC_MAX_CELLS)
        return fail(LB_E_INVAL, "grid has more cells than LB_NOALLOC_MAX_CELLS; use lb_fields with a workspace");
    if (!(eos->a > 0 && eos->b > 0 && eos->R > 0 && eos->G < 0) || !(th->Ts_over_Tc > 0 && th->Ts_over_Tc < 1))
        return fail(LB_E_INVAL, "bad EOS or thermal parameters");

    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return fail(LB_E_CUDA, cudaGetErrorString(e));
    Acc* acc = (Acc*)base;
    float* planes = (float*)((unsigned char*)base + kAccBytes);

    // parameters of the pulled populations, the equation of state and the
    // forces at this level; the arrays are unpitched [.][Ly][Lx]
    StepParams P;
    memset(&P, 0, sizeof(P));
    const double Tc = 0.0778 * eos->a / (0.45724 * eos->b * eos->R);
    const double kappa = 0.37464 + 1.54226 * eos->omega - 0.26992 * eos->omega * eos->omega;
    P.f_in = fpost;
    P.th_in = theta;
    P.acc = acc;
    P.Lx = grid->Lx;
    P.Ly = grid->Ly;
    P.pitch = grid->Lx;
    P.plane = (int)cells;
    P.bc = grid->bc_y;
    P.ghost = grid->ghost_layer ? 1 : 0;
    P.Ts = (float)(th->Ts_over_Tc * Tc);
    P.a = (float)eos->a;
    P.b = (float)eos->b;
    P.R = (float)eos->R;
    P.G = (float)eos->G;
    P.two_over_G = (float)(2.0 / eos->G);
    P.k0 = (float)(1.0 + kappa);
    P.k1 = (float)(kappa / sqrt(Tc));
    P.g = (float)th->g;
    P.rho_ave = (float)rho_ave;
    P.gw6 = (float)(Gw / 6.0);

    // the fault flags must start at zero; the planes are fully rewritten
    e = cudaMemsetAsync(acc, 0, sizeof(Acc), st);
    if (e == cudaSuccess) e = launch_macro(P, planes, rho, ux, uy, T, grid->Lx, st);
    unsigned flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, &acc->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(LB_E_CUDA, cudaGetErrorString(e));
    if (flags & ERR_EOS) return fail(LB_E_EOS_DOMAIN, "pseudopotential argument 2(p - rho/3)/G < 0 (EOS domain)");
    return LB_OK;
}
