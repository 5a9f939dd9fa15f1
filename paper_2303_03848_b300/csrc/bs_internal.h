// bs_internal.h -- host-side declarations shared by the translation units of
// the library (launch wrappers and their argument blocks).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bs_common.cuh"

namespace bsp {

// Arguments of the slice propagation kernel (fine or coarse over all slices).
struct PropArgs {
  enum Mode { kPlain = 0, kPinnFused = 1 };
  const Inst* insts;
  const int32_t* ids;        // instances of this partition class
  const double* pool;        // coefficient blocks
  const double* exptab;      // exp(-r m dtau) tables
  const double* in;          // input states
  double* out;               // outputs
  int in_state;              // 1: input slice n at state_off + n*Nx; 0: at slice_off + n*Nx
  int out_state;             // 1: output at state_off + (n+1)*Nx; 0: at slice_off + n*Nx
  int mode;
  int k_iter;                // Parareal iteration, slices n < k_iter skipped (-1: none)
  const uint8_t* active;     // nullable, per (instance, slice)
  const Ctrl* ctrl;          // nullable, done flags
  const double* uold;        // kPinnFused: U^k (state layout)
  double* normbuf;           // kPinnFused: (num, den) per (instance, boundary index, cluster rank)
  int* status;               // nullable: BS_TIMEOUT recorded here if a bounded wait gave up
  int* task_ctr;             // nullable, zero at launch: one-CTA grids take their tasks from this counter
  const int* n_live;         // nullable: instances not yet converged; the launch does nothing when 0
  int n_inst, maxP;          // tasks = n_inst x ceil((maxP - max(k_iter, 0)) / S2), set by launch_prop
};

struct SerialArgs {
  const Inst* insts;
  const int32_t* ids;
  const double* pool;
  const double* exptab;
  double* out;  // state layout
  int* status;  // nullable: BS_TIMEOUT recorded here if a bounded wait gave up
};

struct SweepArgs {
  const Inst* insts;
  const int32_t* ids;
  const double* pool;
  const double* exptab;
  int kind;            // 0 implicit Euler, 1 network increment, 2 network-anchored implicit Euler
  int k_iter;          // -1: initial sweep
  const Ctrl* ctrl;
  const double* ucur;  // U^k (state layout)
  double* unext;       // U^{k+1} (state layout)
  double* gold;        // G(U^k_n) per slice (slice layout), updated in place
  const double* fbuf;  // F(U^k_n) (slice layout)
  const double* gtab;  // network table (state layout), increment kind; corrections c_n, anchored kind
  double* normbuf;
  int* status;         // nullable: BS_TIMEOUT recorded here if a bounded wait gave up
  const int* n_live;   // nullable: instances not yet converged; the launch does nothing when 0
};

bool partition_supported(int M, int NW, int C);
cudaError_t launch_setup(const Inst* d_insts, const int32_t* d_ids, int n, int Ws, double* pool, double* exptab,
                         cudaStream_t s);
// Persistent propagation launch; s2 = 2 runs two slices of an instance per CTA
// (fine propagator, classes with s2_supported only).
bool s2_supported(int M, int NW, int C);
cudaError_t launch_prop(int M, int NW, int C, int s2, bool cn, const PropArgs& a, int n_inst, int maxP,
                        cudaStream_t s);
cudaError_t launch_serial(int M, int NW, int C, const SerialArgs& a, int n_inst, cudaStream_t s);
cudaError_t launch_sweep(int M, int NW, int C, const SweepArgs& a, int n_inst, cudaStream_t s);
cudaError_t launch_parareal_init(const Inst* d_insts, int n_inst, double* buf0, double* buf1, const double* gtab,
                                 int pinn, Ctrl* ctrl, double* norms, int max_iter, cudaStream_t s);
cudaError_t launch_parareal_finalize(const Inst* d_insts, int n_inst, const double* normbuf, int k, double tol,
                                     int max_iter, Ctrl* ctrl, double* norms, int* live_out, cudaStream_t s);
cudaError_t launch_copy_result(const Inst* d_insts, int n_inst, const Ctrl* ctrl, const double* buf0,
                               const double* buf1, double* out, cudaStream_t s);
cudaError_t launch_grid_points(const Inst* d_insts, int n_inst, int d_in, double* X, cudaStream_t s);
cudaError_t launch_table_fix(const Inst* d_insts, int n_inst, const double* exptab, double* g, cudaStream_t s);
// Network-anchored IE: table slots 1..P become c_n = g_{n+1} - IE(g_n) (gie: IE(g_n), slice layout).
cudaError_t launch_table_correction(const Inst* d_insts, int n_inst, const double* gie, double* g, cudaStream_t s);

// ---- network (pinn.cu) ----
struct MlpDev {
  int n_lin;
  int d_in;
  int max_w;
  int32_t widths[16];
  int64_t poff[16];          // parameter offset of layer l (1-based), in elements
  double lo[8], hi[8];
  const double* p64;         // FP64 master parameters
  const float* p32;          // FP32 copy
  unsigned char* tc_packed;  // square layers in the tensor-core operand layout (pinn_tc.cu)
  int* status;               // device status word: BS_TIMEOUT if a bounded wait gave up
};

// Tensor-core evaluation (pinn_tc.cu): hidden layers w x w on tcgen05, BF16
// or TF32 operands (tf32), FP32 accumulation.
bool tc_supported(const MlpDev& m);
bool tc_fits(const MlpDev& m, bool tf32);
size_t tc_packed_bytes(const MlpDev& m);
cudaError_t launch_mlp_eval_tc(const MlpDev& m, unsigned char* packed, const double* X, int64_t N, double* u,
                               int* status, cudaStream_t s, bool tf32);

cudaError_t launch_mlp_eval(const MlpDev& m, int prec, const double* X, int64_t N, double* u, double* derivs,
                            cudaStream_t s);
cudaError_t launch_f64_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s);

// Loss terms and gradient (pinn.cu).  loss3 and grad are device buffers.
struct LossArgs {
  const double* X;
  const int8_t* kind;
  int64_t N;
  double K, sigma, r, Smax, smax_over_K;
  int prec;
  const double* y = nullptr;  // values of the kind-4 data points (null: 0)
};
cudaError_t launch_loss_grad(const MlpDev& m, const LossArgs& la, double* loss3, double* grad, void* workspace,
                             size_t ws_bytes, cudaStream_t s);
// Workspace of the training kernels outside the BF16 tensor-core path: 4 N w_l
// elements per layer for the activations act[l] (hidden layers l = 1..n_lin-1)
// and the adjoints dz[l] (l = 1..n_lin; dz of the output layer: the seeds).
// The CUDA-core kernels keep a layer as rows (p, s) of w_l neurons; the TF32
// tensor-core kernels as blocks of 32 rows, neuron-major inside a block, for
// the batch padded to 32 points.
struct TrainLayout {
  int64_t act_off[16];  // offsets (elements) of act[l], l = 1..n_lin-1
  int64_t dz_off[16];   // offsets of dz[l], l = 1..n_lin
  int64_t total;        // elements
};
// The loss gradient with TF32 operands on tcgen05 (pinn_train_tf32.cu):
// networks d_in (2 or 5) -> w x ... x w -> 1 with w in {32, 64, 96, 128} and
// at least one w x w layer.  ws: FP32 workspace, 16-byte aligned, with TL the
// layout above for the batch padded to a multiple of 32 points; pack:
// train_tf32_pack_bytes(m) bytes (16-byte aligned) for W_l and W_l^T of the
// square layers; cnt: the points per loss term (already counted); grad zeroed
// by the caller, the loss sums go to loss_acc.
bool train_tf32_supported(const MlpDev& m);
size_t train_tf32_pack_bytes(const MlpDev& m);
cudaError_t launch_train_tf32(const MlpDev& m, const LossArgs& la, float* ws, const TrainLayout& TL,
                              unsigned char* pack, const unsigned long long* cnt, double* loss_acc, double* grad,
                              cudaStream_t s);
size_t loss_grad_workspace_bytes(const MlpDev& m, int64_t N);
// The loss gradient on tcgen05 (pinn_train_tc.cu), BF16 operands with FP32
// accumulation: forward with the derivative streams, adjoint and every layer's
// weight gradient for networks d_in (2 or 5) -> w x ... x w -> 1 with w in
// {32, 64, 96, 128}.  The workspace holds the per-layer activations, adjoints
// and partial sums (train_tc_workspace_bytes, 256-byte aligned).  One prepass
// zeroes grad and counts each loss term's points into cnt; the loss sums go to
// loss_acc (3 doubles) and the loss terms (sum / count) to loss3.  The caller
// zeroes cnt and loss_acc.
bool train_tc_supported(const MlpDev& m);
size_t train_tc_workspace_bytes(const MlpDev& m, int64_t N);
cudaError_t launch_train_tc(const MlpDev& m, const LossArgs& la, unsigned char* ws, unsigned long long* cnt,
                            double* loss_acc, double* grad, double* loss3, cudaStream_t s);
// A bounded mbarrier wait that expires (arrive == 0) or completes (pinn_tc.cu).
cudaError_t launch_wait_probe(int arrive, long long limit, int* status, cudaStream_t s);
cudaError_t launch_adam(int64_t n, double* theta, double* mom1, double* mom2, const double* g, int step, double lr,
                        float* p32, cudaStream_t s);

}  // namespace bsp
