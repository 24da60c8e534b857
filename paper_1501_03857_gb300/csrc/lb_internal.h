// Host-side declarations shared by the translation units of liblbboil.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lb_device.cuh"

namespace lbgpu {

// Launch shape of the fused step (lb_step3.cu): block_x threads per block,
// each thread owning one column of two strips of block_x - 2*HALO output
// columns; seg_rows rows per block; nstrips x nseg blocks.
struct Launch {
    int block_x, seg_rows, nstrips, nseg;
};

// One step of the fused kernel: one row per iteration, two column strips per
// block in paired FP32 (block_x 64, 128 or 256).
bool dual_supported(int block_x);
cudaError_t dual_prepare();  // opt in to the dynamic shared memory
cudaError_t dual_occupancy(int block_x, int* blocks_per_sm);
cudaError_t launch_step(const StepParams& P, const Launch& L, cudaStream_t st);

// The forward intermediates of one step that the adjoint's reverse kernels
// read (lb_adjoint.cu), written by the dual-strip step in its recompute mode
// (lb_step3.cu) into pitched [Ly][pitch] planes. The gradients drx, dry and
// div v carry the stencil weights; ax, ay are coefficients of K(T), Eq. 18
// (0 on the wall rows; cA, cB and F_m follow from div v, rho and psi); u2-u4
// the RK stage inputs (theta on the wall rows). With out the step itself is written too (f*, theta of the
// next level to P.f_out, P.th_out), and with heat (only with out) q(t) is
// added to P.acc's heat-flux sums as the plain step does.
struct RecomputeOut {
    float *rho, *psi;
    float *drx, *dry, *divv, *ax, *ay, *u2, *u3, *u4;
};
constexpr int kRecomputePlanes = 10;  // the planes of RecomputeOut, in its order
cudaError_t dual_recompute(const StepParams& P, const RecomputeOut& R, bool out, bool heat, const Launch& L,
                           cudaStream_t st);

// The same step over a table of independent instances in one launch
// (paired FP32, block_x 64 or 128); instance i owns blocks
// [block_off[i], block_off[i+1]).
bool batch_supported(int block_x);
cudaError_t batch_prepare();
cudaError_t batch_occupancy(int block_x, bool shared_k, int* blocks_per_sm);
// K non-null: every instance shares the model constants in *K (see
// step_body in lb_step3.cu) and the kernel reads them from its parameters.
cudaError_t batch_launch(int block_x, const StepParams* table, const int* block_off, int n, int nblocks,
                         const StepParams* K, cudaStream_t st);

// The persistent batch (lb_batch_persist in lb_step3.cu): one cooperative
// launch of a fixed grid advances every instance by nsteps steps; block g
// takes tiles tile_off[g] .. tile_off[g+1]-1 (instance, block index within
// the instance) every step, after all tiles of the instance finished the
// previous step (arrive[i] counts finished tiles of instance i since the
// launch began and must be zero at launch). A wait gives up after
// wait_limit polls, sets ERR_TIMEOUT in the instance's fault flags and ends
// the block.
struct PersistArgs {
    const StepParams* table;  // [2][n], by step parity
    const int2* tiles;
    const int* tile_off;
    const int* ntiles;        // [n] tiles per instance
    unsigned* arrive;         // [n]
    int n, nsteps;
    unsigned long long wait_limit;
};
cudaError_t persist_occupancy(int block_x, bool shared_k, int* blocks_per_sm);
cudaError_t persist_launch(int block_x, const StepParams* K, const PersistArgs& A, int nblocks, cudaStream_t st);

// Initial state: f* = w_a rho0 (rest equilibrium), theta = 0 with the wall
// rows at their Dirichlet values. rho0 is pitched [Ly][pitch].
cudaError_t launch_init(const StepParams& P, const float* rho0, float* f, float* th, cudaStream_t st);

// Macroscopic fields (rho, u with the level's forces, T) into outputs with
// row stride ostride; scratch holds 4 pitched planes.
cudaError_t launch_macro(const StepParams& P, float* scratch, float* rho, float* ux, float* uy,
                         float* T, int ostride, cudaStream_t st);

// Discrete adjoint of one step (lb_adjoint.cu): work bytes, reset of the
// FP64 gradient accumulators, one reverse step, and the final read-out
// (which adds the initial wall row's lambda_theta to dJ/d theta_b).
size_t adjoint_work_bytes(const StepParams& P);
cudaError_t adjoint_grads_reset(const StepParams& P, void* work, cudaStream_t st);
// The adjoint of f* travels between reverse steps in two parts: lambda of
// f*_a at cell t is lf[a](t) + lr(t + e_a), where lr is one plane (lambda of
// rho = sum f at the cell that pulls f*_a(t); 0 outside the domain and on
// the wall rows and the outflow top, whose share is already in lf). Zero lf
// and lr are a zero adjoint. The in and out planes are distinct buffers.
// R holds the forward intermediates of the step being reversed (written by
// dual_recompute from the same state).
cudaError_t adjoint_reverse_step(const StepParams& P, const RecomputeOut& R, void* work, const float* fstar,
                                 const float* theta, const float* lf_in, const float* lt_in, const float* lr_in,
                                 float* lf_out, float* lt_out, float* lr_out, float lq, cudaStream_t st);
cudaError_t adjoint_grads_finish(const StepParams& P, void* work, const float* lt0, double* dTb_host,
                                 double* dGw_host, cudaStream_t st);

// Record the message lb_last_error() returns on this thread.
void set_last_error(const char* msg);

// acc->mass = sum over cells and directions of f (FP64).
cudaError_t launch_mass(const StepParams& P, const float* f, cudaStream_t st);

// Pressure probes (Fig. 3): after a step, record (rho^t, T^t, p_EOS) at up to
// kProbeMax cells into a device ring (256-byte header whose first 8 bytes
// count the probed steps, then float4 records [probe][cap]).
constexpr int kProbeMax = 8;
struct ProbeArgs {
    const float* f;   // post-collision populations written by the step (level t)
    const float* th;  // theta^t, the step's input temperature
    float* ring;
    int plane, pitch, n, cap;
    int x[kProbeMax], y[kProbeMax];
    double a, b, R, Ts, k0, k1;  // Eq. 21: phi(T) = (k0 - k1 sqrt(T))^2
};
cudaError_t launch_probe(const ProbeArgs& A, cudaStream_t st);

}  // namespace lbgpu
