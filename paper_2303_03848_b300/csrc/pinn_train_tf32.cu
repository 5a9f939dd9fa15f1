// pinn_train_tf32.cu -- the loss gradient of one training step (Section 3.3,
// the loss of Eqs. 11-14 and its adjoint) with TF32 operands on the tensor
// cores: FP32 values rounded to TF32 (cvt.rna), FP32 accumulation in tensor
// memory (tcgen05.mma kind::tf32).
//
// A tile is 128 rows (p, s), row 4 p + s for 32 points p and the derivative
// streams s = 0 value, 1 d/dS, 2 d2/dS2, 3 d/dtau.  The four streams of a
// layer share its weights, so one M = 128 GEMM per layer covers all of them,
// and the four rows of a point sit on four adjacent lanes of one warp, which
// exchange by shuffles what couples the streams:
//   forward   z_s = W h_s (+ b on the value rows), t = tanh z_0, t' = 1 - t^2,
//             h_0 = t, h_1 = t' z_1, h_2 = t' (z_2 - 2 t z_1^2), h_3 = t' z_3;
//   adjoint   ah_s = W^T dz_s (rank one from the loss seeds at the top), then
//             dz_s = t' X_s with X_0 = ah_0 - 2 t' b2 - 2 t (b1 - 2 t b2),
//             b2 = ah_2 z_1^2, b1 = ah_1 z_1 + ah_2 z_2 + ah_3 z_3,
//             X_1 = ah_1 - 4 t ah_2 z_1, X_2 = ah_2, X_3 = ah_3;
//   gradient  dL/dW[o][i] = sum over rows of dz[row][o] h[row][i] and
//             dL/db[o] = sum over value rows of dz[row][o].
// Workspace (FP32): act[l] (hidden layers) holds per neuron o and row (p, s)
// the value t for s = 0 and z_s for s > 0; dz[l] the adjoint of every layer
// (the output layer's: the seeds).  Both are blocked and neuron-major: the
// 32 rows of block b for neuron o at (b w_l + o) 32, so a warp's 32 lanes
// (one block) store one neuron as one 128-byte line, a tile's layer is 4
// consecutive blocks (the adjoint fetches them with one bulk copy), a point's
// four values are one 16-byte load, and a stage of the weight gradient reads
// one contiguous block per operand.  The batch is padded to whole tiles.
// Three kernels:
//   train_tf32_fwd_kernel   input layer on CUDA cores, the square layers on
//                           the tensor cores (W_l staged by TMA), output layer,
//                           loss terms and seeds on CUDA cores;
//   train_tf32_bwd_kernel   the adjoint top down against the packed W_l^T;
//   train_tf32_wgrad_kernel every layer's weight and bias gradient as one GEMM
//                           with K = rows: A = dz_l^T (M = neurons o), B =
//                           h_{l-1}^T (N = inputs i, plus one column that is 1
//                           on value rows: the bias), h rebuilt from act.
// Every mbarrier wait is bounded: on expiry a kernel records BS_TIMEOUT,
// waits (bounded) for its copy in flight, frees its tensor memory and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "bs_common.cuh"
#include "bs_internal.h"
#include "pinn_loss.cuh"
#include "tcgen05.cuh"

namespace bsp {

using namespace tc;

namespace {

constexpr int kT32Rows = 128;  // rows of a tile (TMEM lanes)
constexpr int kT32Pts = 32;    // points of a tile
constexpr int kBlk = 32;       // rows of a block of the workspace layout
constexpr int kWgK = 32;       // rows (K) per stage of the weight gradient: one block
constexpr int kWgRaw = 2;      // its raw-block buffers (stages in flight)
constexpr int kWgOps = 1;      // its operand buffers

__device__ __forceinline__ float tf32r(float x) { return __uint_as_float(to_tf32(x)); }

struct T32Args {
  MlpDev m;
  LossArgs la;
  float* ws;
  int64_t act_off[16], dz_off[16];
  const unsigned char* wfwd;  // W_l, l = 2 .. n_lin-1: [l - 2] w x w (rows o, K = i), TF32 core matrices
  const unsigned char* wbwd;  // W_l^T: [l - 2] w x w (rows i, K = o)
  const unsigned long long* cnt;
  double* loss_acc;
  int ntiles;
};

// Square layers packed as B operands: W_l (rows o, K = i) for the forward and
// W_l^T (rows i, K = o) for the adjoint, TF32 (cvt.rna) in the no-swizzle
// K-major core-matrix layout.
__global__ void pack_tf32_train_kernel(MlpDev m, int w, unsigned char* fwd, unsigned char* bwd) {
  const int n_sq = m.n_lin - 2;
  const int64_t per = (int64_t)w * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * n_sq;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / per);
    const int o = (int)((e % per) / w), i = (int)(e % w);
    const uint32_t v = to_tf32(m.p32[m.poff[q + 2] + (int64_t)o * w + i]);
    *reinterpret_cast<uint32_t*>(fwd + q * per * 4 + canon_off_eb<4>(o, i, w)) = v;
    *reinterpret_cast<uint32_t*>(bwd + q * per * 4 + canon_off_eb<4>(i, o, w)) = v;
  }
}

// Input map of coordinate k to [-1, 1] as the forward uses it: x^ = sc x + of
// in FP32 (the result is rounded to TF32).
struct InMap {
  float sc[8], of[8];
};

// Entry k of the map (thread k of a CTA fills the CTA's shared copy).
__device__ __forceinline__ void inmap_entry(const MlpDev& m, int k, InMap& im) {
  if (k < m.d_in) {
    const double g = 2.0 / (m.hi[k] - m.lo[k]);
    im.sc[k] = (float)g;
    im.of[k] = (float)(-g * m.lo[k] - 1.0);
  } else {
    im.sc[k] = 0.0f;
    im.of[k] = 0.0f;
  }
}

// Stream s of input coordinate k at point p (x^ on the value row, d x^ / dS
// and d x^ / dtau on rows 1 and 3), TF32-rounded.
template <int DIN>
__device__ __forceinline__ float input_stream(const InMap& im, const double* X, int64_t p, int s, int k) {
  if (s == 0) return tf32r(fmaf(im.sc[k], (float)X[p * DIN + k], im.of[k]));
  if (s == 1) return k == 0 ? tf32r(im.sc[0]) : 0.0f;
  if (s == 3) return k == 1 ? tf32r(im.sc[1]) : 0.0f;
  return 0.0f;
}

// The weights of the next GEMM have landed (thread 0; bounded).
__device__ __forceinline__ void wait_weights(bool& pending, uint32_t& ph, uint64_t* bar, int* fail) {
  if (pending) {
    if (mbar_wait_bounded(bar, ph)) {
      ph ^= 1u;
      pending = false;
    } else {
      *fail = 1;
    }
  }
}

// One square-layer GEMM: D (TMEM, 128 x n) = A (128 x w, sA) x B^T (n x w, sB),
// w / 8 MMAs of K = 8, committed to bar (thread 0).
__device__ __forceinline__ void issue_gemm_tf32(uint32_t tmem, const unsigned char* sA, const unsigned char* sB, int w,
                                                int n, uint64_t* bar) {
  const uint32_t aa = smem_u32(sA), bb = smem_u32(sB), sbo = (uint32_t)(w / 4) * 128;
  const uint32_t idesc = make_idesc_tf32(n);
  for (int kk = 0; kk < w / 8; ++kk)
    mma_tf32(tmem, make_desc(aa + kk * 256, 128, sbo), make_desc(bb + kk * 256, 128, sbo), idesc, kk > 0 ? 1u : 0u);
  mma_commit(bar);
}

// Shared memory of the forward and adjoint kernels: the B operand (one layer's
// W_l or W_l^T), the 128 x w A operand, the input layer (w x d_in, TF32), the
// hidden biases, the output weights (TF32), the output partial sums of the w / 32
// column groups, two mbarriers and the tensor-memory address.
__host__ __device__ constexpr size_t t32_smem_bytes(int w, int din, int n_lin) {
  return (size_t)w * w * 4 + (size_t)kT32Rows * w * 4 +
         4 * ((size_t)w * din + (size_t)(n_lin - 1) * w + w + (size_t)(w / 32) * kT32Rows) + 32;
}

// Forward of a training step.  CTA: 4 w threads; warp v reads accumulator lanes
// 32 (v % 4) .. + 31 (one row each) and owns columns 32 (v / 4) .. + 31.
template <int DIN, int W>
__global__ void __launch_bounds__(4 * W, 1) train_tf32_fwd_kernel(T32Args a) {
  constexpr int NG = W / 32;
  constexpr uint32_t WB = W * W * 4, AB = kT32Rows * W * 4;
  constexpr uint32_t NCOLS = W <= 32 ? 32 : (W <= 64 ? 64 : 128);
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int n_lin = m.n_lin, L = n_lin - 1, n_sq = n_lin - 2;
  unsigned char* sW = smem;
  unsigned char* sA = smem + WB;
  float* sW1 = reinterpret_cast<float*>(sA + AB);  // [W][DIN]
  float* sB = sW1 + W * DIN;                        // [L][W] biases of hidden layers 1..L
  float* sWo = sB + L * W;                          // [W]
  float* sred = sWo + W;                            // [NG][128]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sred + NG * kT32Rows);  // [0] MMAs done, [1] weights landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int s_fail;
  __shared__ double s_acc[3];
  __shared__ float s_icnt[3];
  __shared__ InMap s_im;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, qd = warp & 3, g = warp >> 2;
  const int r = qd * 32 + lane, s = r & 3, pl = r >> 2, c0 = g * 32, base = lane & ~3;
  const int64_t N = a.la.N;
  if (t < 8) inmap_entry(m, t, s_im);
  for (int i = t; i < W * DIN; i += blockDim.x) sW1[i] = tf32r(m.p32[m.poff[1] + i]);
  for (int i = t; i < L * W; i += blockDim.x) {
    const int l = i / W + 1, o = i % W;
    sB[i] = m.p32[m.poff[l] + (int64_t)W * m.widths[l - 1] + o];
  }
  for (int o = t; o < W; o += blockDim.x) sWo[o] = tf32r(m.p32[m.poff[n_lin] + o]);
  const float bout = m.p32[m.poff[n_lin] + W];
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    s_acc[0] = s_acc[1] = s_acc[2] = 0.0;
    for (int k = 0; k < 3; ++k) s_icnt[k] = a.cnt[k] ? 1.0f / (float)a.cnt[k] : 0.0f;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool w_pending = false;
  uint32_t ph_w = 0, ph_mma = 0;
  if (t == 0 && (int)blockIdx.x < a.ntiles) {
    bulk_load(sW, a.wfwd, WB, &bar[1]);
    w_pending = true;
  }
  if (warp == 0) tmem_alloc(tslot, NCOLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tl = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0;
  const float bm = s == 0 ? 1.0f : 0.0f;  // the bias enters the value rows only
  float sqs[3] = {0.0f, 0.0f, 0.0f};

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const bool last_tile = tile + (int)gridDim.x >= a.ntiles;
    const int64_t p = (int64_t)tile * kT32Pts + pl;
    const bool live = p < N;
    float z[32];
    {  // input layer on CUDA cores
      float hin[DIN];
#pragma unroll
      for (int k = 0; k < DIN; ++k) hin[k] = live ? input_stream<DIN>(s_im, a.la.X, p, s, k) : 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < DIN; ++k) acc = fmaf(hin[k], sW1[(c0 + j) * DIN + k], acc);
        z[j] = fmaf(bm, sB[c0 + j], acc);
      }
    }
    float dot = 0.0f;  // output layer: this thread's part of W_out h_s
    // hidden layer l from its pre-activations z: (t, z_1, z_2, z_3) stored,
    // h rounded to TF32 as the next A operand (or into the output dot product)
    auto epilogue = [&](int l, bool top) {
      float* act = a.ws + a.act_off[l] + (int64_t)tile * W * kT32Rows + qd * W * kBlk;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        float hq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float zz = z[j + u];
          const float z0 = __shfl_sync(kFull, zz, base);
          const float z1 = __shfl_sync(kFull, zz, base + 1);
          const float tt = tanh_fast(z0), d1 = 1.0f - tt * tt;
          const float inner = s == 2 ? fmaf(-2.0f * tt * z1, z1, zz) : zz;
          if (live) act[(c0 + j + u) * kBlk + lane] = s == 0 ? tt : zz;
          hq[u] = tf32r(s == 0 ? tt : d1 * inner);
        }
        if (top) {
          const float4 wq = *reinterpret_cast<const float4*>(sWo + c0 + j);
          dot = fmaf(wq.x, hq[0], dot);
          dot = fmaf(wq.y, hq[1], dot);
          dot = fmaf(wq.z, hq[2], dot);
          dot = fmaf(wq.w, hq[3], dot);
        } else {
          *reinterpret_cast<float4*>(sA + canon_off_eb<4>(r, c0 + j, W)) = make_float4(hq[0], hq[1], hq[2], hq[3]);
        }
      }
    };
    epilogue(1, false);
    for (int q = 0; q < n_sq; ++q) {  // square layer l = q + 2
      fence_proxy_async();            // the A operand's generic-proxy writes visible to the tensor core
      fence_before();
      __syncthreads();
      fence_after();
      if (t == 0) {
        wait_weights(w_pending, ph_w, &bar[1], &s_fail);
        if (!s_fail) {
          issue_gemm_tf32(tmem, sA, sW, W, W, &bar[0]);
          if (!mbar_wait_bounded(&bar[0], ph_mma)) {
            s_fail = 1;
          } else if (!(last_tile && q == n_sq - 1)) {  // the next weights load while the epilogue runs
            const int nxt = q + 1 < n_sq ? q + 1 : 0;
            bulk_load(sW, a.wfwd + (size_t)nxt * WB, WB, &bar[1]);
            w_pending = true;
          }
        }
      }
      ph_mma ^= 1u;
      fence_before();
      __syncthreads();
      fence_after();
      if (s_fail) break;
      {
        float v[32];
        tmem_ld32(tl, v);
        const float* bl = sB + (q + 1) * W + c0;
#pragma unroll
        for (int j = 0; j < 32; ++j) z[j] = fmaf(bm, bl[j], v[j]);
      }
      epilogue(q + 2, q == n_sq - 1);
      fence_before();  // accumulator reads done before the next MMA overwrites it
    }
    if (s_fail) break;
    // output streams of the tile's rows, then loss terms and seeds per point
    sred[g * kT32Rows + r] = dot;
    __syncthreads();
    if (g == 0) {
      float out = s == 0 ? bout : 0.0f;
#pragma unroll
      for (int q = 0; q < NG; ++q) out += sred[q * kT32Rows + r];
      float o4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) o4[u] = __shfl_sync(kFull, out, base + u);
      if (s == 0 && live) {
        const int kd = a.la.kind[p];
        float x[8];
#pragma unroll
        for (int k = 0; k < DIN; ++k) x[k] = (float)a.la.X[p * DIN + k];
        const float yv = (kd == 4 && a.la.y != nullptr) ? (float)a.la.y[p] : 0.0f;
        const float ic[3] = {s_icnt[0], s_icnt[1], s_icnt[2]};
        float sq[3] = {0.0f, 0.0f, 0.0f}, gq[4];
        point_loss_f32(a.la, DIN, x, kd, yv, o4, ic, sq, gq);
        sqs[0] += sq[0];
        sqs[1] += sq[1];
        sqs[2] += sq[2];
        *reinterpret_cast<float4*>(a.ws + a.dz_off[n_lin] + 4 * p) = make_float4(gq[0], gq[1], gq[2], gq[3]);
      }
    }
  }
  // loss sums: warp, CTA, then the call's accumulators
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float v = sqs[k];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0 && v != 0.0f) atomicAdd(&s_acc[k], (double)v);
  }
  if (t == 0 && w_pending) (void)mbar_wait_bounded(&bar[1], ph_w);  // a copy in flight lands before exit
  fence_before();
  __syncthreads();
  fence_after();
  if (t == 0) {
    if (s_fail) atomicExch(m.status, 6);  // BS_TIMEOUT
    for (int k = 0; k < 3; ++k)
      if (s_acc[k] != 0.0) atomicAdd(a.loss_acc + k, s_acc[k]);
  }
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// Shared memory of the adjoint: the B operand (W_l^T), the 128 x w A operand,
// the tile's stored activations of one layer ([w][128] FP32, filled by TMA
// bulk copies), the output weights, three mbarriers and the TMEM address.
__host__ __device__ constexpr size_t t32_bwd_smem_bytes(int w) {
  return (size_t)w * w * 4 + 2 * (size_t)kT32Rows * w * 4 + 4 * (size_t)w + 64;
}

// Adjoint of a training step on the same tiles, top layer down: ah of layer L
// from the seeds (rank one, CUDA cores), then per layer l the stored
// (t, z_1, z_2, z_3) turn ah into dz_l (stored), and for l >= 2 the GEMM
// dz_l W_l (B = the packed W_l^T) gives ah of layer l - 1.  The activations of
// the next layer down come into shared memory (one 512-byte bulk copy per
// neuron: its 128 rows of the tile) while that GEMM runs.
template <int DIN, int W>
__global__ void __launch_bounds__(4 * W, 1) train_tf32_bwd_kernel(T32Args a) {
  constexpr uint32_t WB = W * W * 4, AB = kT32Rows * W * 4;
  constexpr uint32_t NCOLS = W <= 32 ? 32 : (W <= 64 ? 64 : 128);
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int n_lin = m.n_lin, L = n_lin - 1;
  unsigned char* sW = smem;
  unsigned char* sA = smem + WB;
  float* sAct = reinterpret_cast<float*>(sA + AB);  // [4][W][32]: the tile's 4 blocks
  float* sWo = sAct + W * kT32Rows;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sWo + W);  // [0] MMAs done, [1] weights, [2] activations
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
  __shared__ int s_fail;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, qd = warp & 3, g = warp >> 2;
  const int r = qd * 32 + lane, s = r & 3, pl = r >> 2, c0 = g * 32, base = lane & ~3;
  const int64_t N = a.la.N;
  for (int o = t; o < W; o += blockDim.x) sWo[o] = tf32r(m.p32[m.poff[n_lin] + o]);
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // B operand of the GEMM below layer l (l = L .. 2): W_l^T
  auto wsrc = [&](int l) { return a.wbwd + (size_t)(l - 2) * WB; };
  // thread 0: the tile's 4 blocks of act[l] into sAct
  auto fetch_act = [&](int l, int tile) {
    bulk_load(sAct, a.ws + a.act_off[l] + (int64_t)tile * W * kT32Rows, AB, &bar[2]);
  };
  bool w_pending = false, act_pending = false;
  uint32_t ph_w = 0, ph_mma = 0, ph_act = 0;
  if (t == 0 && (int)blockIdx.x < a.ntiles) {
    bulk_load(sW, wsrc(L), WB, &bar[1]);
    w_pending = true;
  }
  if (warp == 0) tmem_alloc(tslot, NCOLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tl = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)c0;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    __syncthreads();  // the previous tile's reads of sAct are done
    if (s_fail) break;
    const bool last_tile = tile + (int)gridDim.x >= a.ntiles;
    const int64_t p = (int64_t)tile * kT32Pts + pl;
    const bool live = p < N;
    const int64_t row = 4 * p + s;
    if (t == 0) fetch_act(L, tile);
    act_pending = true;
    float ah[32];
    {
      const float sd = live ? tf32r(a.ws[a.dz_off[n_lin] + row]) : 0.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) ah[j] = sWo[c0 + j] * sd;
    }
    for (int l = L; l >= 1; --l) {
      // this layer's activations have landed (every thread waits, bounded)
      if (!mbar_wait_bounded(&bar[2], ph_act)) s_fail = 1;
      ph_act ^= 1u;
      act_pending = false;
      float* dzl = a.ws + a.dz_off[l] + (int64_t)tile * W * kT32Rows + qd * W * kBlk;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        float gq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = c0 + j + u;
          float4 av = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          if (live) av = *reinterpret_cast<const float4*>(sAct + (qd * W + i) * kBlk + (lane & ~3));
          const float own = ah[j + u];
          const float ahS = __shfl_sync(kFull, own, base + 1);
          const float ahSS = __shfl_sync(kFull, own, base + 2);
          const float ahT = __shfl_sync(kFull, own, base + 3);
          const float tt = av.x, zs = av.y, zss = av.z, zt = av.w;
          const float d1 = 1.0f - tt * tt;
          const float b2 = ahSS * zs * zs;
          const float b1 = fmaf(-2.0f * tt, b2, fmaf(ahS, zs, fmaf(ahSS, zss, ahT * zt)));
          const float x0 = fmaf(-2.0f * tt, b1, fmaf(-2.0f * d1, b2, own));
          const float x1 = fmaf(-4.0f * tt * ahSS, zs, own);
          const float gv = live ? d1 * (s == 0 ? x0 : (s == 1 ? x1 : own)) : 0.0f;
          if (live) dzl[i * kBlk + lane] = gv;
          gq[u] = tf32r(gv);
        }
        if (l >= 2)
          *reinterpret_cast<float4*>(sA + canon_off_eb<4>(r, c0 + j, W)) = make_float4(gq[0], gq[1], gq[2], gq[3]);
      }
      if (l == 1) break;
      fence_proxy_async();
      fence_before();
      __syncthreads();  // sA complete; this layer's sAct reads done
      fence_after();
      if (s_fail) break;
      if (t == 0) fetch_act(l - 1, tile);  // overlaps the GEMM below
      act_pending = true;
      if (t == 0) {
        wait_weights(w_pending, ph_w, &bar[1], &s_fail);
        if (!s_fail) {
          issue_gemm_tf32(tmem, sA, sW, W, W, &bar[0]);
          if (!mbar_wait_bounded(&bar[0], ph_mma)) {
            s_fail = 1;
          } else if (!(last_tile && l == 2)) {
            bulk_load(sW, wsrc(l > 2 ? l - 1 : L), WB, &bar[1]);
            w_pending = true;
          }
        }
      }
      ph_mma ^= 1u;
      fence_before();
      __syncthreads();
      fence_after();
      if (s_fail) break;
      tmem_ld32(tl, ah);
      fence_before();
    }
  }
  // copies still in flight (only after a failed wait) land before exit
  if (act_pending && !mbar_wait_bounded(&bar[2], ph_act)) s_fail = 1;
  if (t == 0 && w_pending) (void)mbar_wait_bounded(&bar[1], ph_w);
  fence_before();
  __syncthreads();
  fence_after();
  if (t == 0 && s_fail) atomicExch(m.status, 6);  // BS_TIMEOUT
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// Weight and bias gradient of every layer l: D[o][n] = sum over the CTA's rows
// of A[o][row] B[n][row] with A = dz_l^T (M = 128 rows o, rows o >= w_l zero)
// and B = h_{l-1}^T (rows n < w_{l-1}; row n = w_{l-1} is 1 on value rows and
// 0 elsewhere, so column w_{l-1} of D is the bias gradient; zero rows pad N to
// a multiple of 16).  A stage is one 32-row block: thread 0 fetches the
// block of dz_l and of act_{l-1} with one bulk copy each, kWgRaw - 1 stages
// ahead; all threads convert a landed block into the K-major core-matrix
// operands (TF32 rounding; h_{l-1} rebuilt from the stored activations exactly
// as the forward formed it, layer 1 from the inputs; rows past the batch
// zero); one thread issues the stage's kWgK / 8 MMAs and commits them to the
// operand buffer's mbarrier.  Each CTA adds its D into the FP64 gradient.
// ---------------------------------------------------------------------------
struct WgT32Args {
  MlpDev m;
  const double* X;
  int64_t N;
  const float* ws;
  int64_t act_off[16], dz_off[16];
  int cta0[18];        // first CTA of layer l (l = 1 .. n_lin); cta0[n_lin + 1] = the grid
  int64_t crows[17];   // rows per CTA of layer l (a multiple of kWgK)
  double* grad;
};

template <int W>
__host__ __device__ constexpr uint32_t wg_ops_bytes() {
  return (uint32_t)kT32Rows * kWgK * 4 + (uint32_t)(W + 16) * kWgK * 4;
}
template <int W>
__host__ __device__ constexpr size_t wg_smem_bytes() {
  return (size_t)kWgRaw * 2 * W * kWgK * 4 + (size_t)kWgOps * wg_ops_bytes<W>() + 8 * (kWgRaw + kWgOps) + 8;
}

template <int DIN, int W>
__global__ void __launch_bounds__(256, 2) train_tf32_wgrad_kernel(WgT32Args a) {
  constexpr uint32_t RAWB = W * kWgK * 4;  // one raw block of W neurons
  constexpr uint32_t ABYTES = kT32Rows * kWgK * 4;
  constexpr uint32_t OPS = wg_ops_bytes<W>();
  constexpr int NBMAX = W + 16;
  constexpr uint32_t NCOLS = NBMAX <= 32 ? 32 : (NBMAX <= 64 ? 64 : (NBMAX <= 128 ? 128 : 256));
  constexpr uint32_t SBO = (kWgK / 4) * 128;
  constexpr int IT = W * (kWgK / 4) / 256;  // pieces (4 rows of one neuron) per thread and operand
  static_assert(IT >= 1 && W * (kWgK / 4) % 256 == 0, "stage pieces must split evenly over 256 threads");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* rawA = smem;                          // [kWgRaw][W][32] dz blocks
  unsigned char* rawB = smem + kWgRaw * RAWB;          // [kWgRaw][W][32] act blocks
  unsigned char* ops = smem + 2 * kWgRaw * RAWB;       // [kWgOps] A, B operands
  uint64_t* rbar = reinterpret_cast<uint64_t*>(ops + kWgOps * OPS);  // [kWgRaw] blocks landed
  uint64_t* obar = rbar + kWgRaw;                                     // [kWgOps] MMAs done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(obar + kWgOps);
  __shared__ int s_fail;
  __shared__ InMap s_im;
  const MlpDev& m = a.m;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  int l = 1;
  while (l < m.n_lin && (int)blockIdx.x >= a.cta0[l + 1]) ++l;
  const int64_t R = 4 * a.N;
  const int64_t rb = (int64_t)((int)blockIdx.x - a.cta0[l]) * a.crows[l];
  const int64_t re = rb + a.crows[l] < R ? rb + a.crows[l] : R;
  const int wo = m.widths[l], wi = m.widths[l - 1];
  const int nb = ((wi + 1 + 15) / 16) * 16;
  const int nst = re > rb ? (int)((re - rb + kWgK - 1) / kWgK) : 0;
  const float* dz = a.ws + a.dz_off[l];
  const float* act = l >= 2 ? a.ws + a.act_off[l - 1] : nullptr;
  if (t == 0) {
    for (int k = 0; k < kWgRaw; ++k) mbar_init(&rbar[k], 1);
    for (int k = 0; k < kWgOps; ++k) mbar_init(&obar[k], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (t < 8) inmap_entry(m, t, s_im);
  // the constant parts of the operands: A rows o >= wo zero; B row wi the bias
  // column, rows wi + 1 .. nb - 1 zero
  for (int k = 0; k < kWgOps; ++k) {
    unsigned char* A = ops + k * OPS;
    unsigned char* B = A + ABYTES;
    for (int e = t; e < (kT32Rows - wo) * kWgK; e += blockDim.x)
      *reinterpret_cast<float*>(A + canon_off_eb<4>(wo + e / kWgK, e % kWgK, kWgK)) = 0.0f;
    for (int e = t; e < (nb - wi) * kWgK; e += blockDim.x) {
      const int n = wi + e / kWgK, kr = e % kWgK;
      *reinterpret_cast<float*>(B + canon_off_eb<4>(n, kr, kWgK)) = (n == wi && (kr & 3) == 0) ? 1.0f : 0.0f;
    }
  }
  if (warp == 0) tmem_alloc(tslot, NCOLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc_tf32(nb);
  // thread 0: the blocks of stage j (its first row rb + 32 j starts a block)
  auto fetch = [&](int j) {
    const int k = j % kWgRaw;
    const int64_t blk = (rb + (int64_t)j * kWgK) / kBlk;
    uint32_t bytes = (uint32_t)wo * kWgK * 4;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&rbar[k])),
                 "r"(bytes + (act != nullptr ? (uint32_t)wi * kWgK * 4 : 0u))
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(rawA + k * RAWB)),
                 "l"(dz + blk * wo * kBlk), "r"(bytes), "r"(smem_u32(&rbar[k]))
                 : "memory");
    if (act != nullptr) {
      bytes = (uint32_t)wi * kWgK * 4;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(rawB + k * RAWB)),
                   "l"(act + blk * wi * kBlk), "r"(bytes), "r"(smem_u32(&rbar[k]))
                   : "memory");
    }
  };
  // piece u of this thread, e = t + 256 u: neuron n = 8 (e >> 6) + i and
  // point q = ((e >> 3) + i) & 7 of the block, i = e & 7: the 8 lanes of a
  // 16-byte phase read 8 different 16-byte columns of the raw block and write
  // 8 different core-matrix rows, so neither side has a bank conflict
  auto convert = [&](int j) {
    const unsigned char* rA = rawA + (j % kWgRaw) * RAWB;
    const unsigned char* rB = rawB + (j % kWgRaw) * RAWB;
    unsigned char* A = ops + (j % kWgOps) * OPS;
    unsigned char* B = A + ABYTES;
    const int64_t r0 = rb + (int64_t)j * kWgK;
#pragma unroll
    for (int u = 0; u < IT; ++u) {
      const int e = t + 256 * u, i = e & 7;
      const int n = ((e >> 6) << 3) | i, q = ((e >> 3) + i) & 7;
      const bool in = r0 + 4 * q < re;
      const uint32_t dst = canon_off_eb<4>(n, 4 * q, kWgK);
      if (n < wo) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (in) v = *reinterpret_cast<const float4*>(rA + n * 128 + q * 16);
        *reinterpret_cast<float4*>(A + dst) = make_float4(tf32r(v.x), tf32r(v.y), tf32r(v.z), tf32r(v.w));
      }
      if (n < wi) {
        float4 h = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (in) {
          if (act != nullptr) {  // (t, z_1, z_2, z_3) -> h as the forward formed it
            const float4 v = *reinterpret_cast<const float4*>(rB + n * 128 + q * 16);
            const float tt = v.x, d1 = 1.0f - tt * tt;
            h = make_float4(tf32r(tt), tf32r(d1 * v.y), tf32r(d1 * fmaf(-2.0f * tt * v.y, v.y, v.z)),
                            tf32r(d1 * v.w));
          } else {  // layer 1: the input streams
            const int64_t p = (r0 >> 2) + q;
            h = make_float4(input_stream<DIN>(s_im, a.X, p, 0, n), input_stream<DIN>(s_im, a.X, p, 1, n), 0.0f,
                            input_stream<DIN>(s_im, a.X, p, 3, n));
          }
        }
        *reinterpret_cast<float4*>(B + dst) = h;
      }
    }
  };
  if (t == 0)
    for (int j = 0; j < kWgRaw - 1 && j < nst; ++j) fetch(j);
  int issued = -1;  // last stage whose MMAs were issued
  for (int j = 0; j < nst; ++j) {
    // the raw buffer of stage j - 1 was converted before the last barrier
    if (t == 0 && j + kWgRaw - 1 < nst) fetch(j + kWgRaw - 1);
    if (!mbar_wait_bounded(&rbar[j % kWgRaw], (uint32_t)((j / kWgRaw) & 1))) s_fail = 1;
    if (j >= kWgOps &&  // the MMAs that read this operand buffer (stage j - kWgOps) are done
        !mbar_wait_bounded(&obar[j % kWgOps], (uint32_t)((j / kWgOps - 1) & 1)))
      s_fail = 1;
    convert(j);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (s_fail) break;
    if (t == 0) {
      const uint32_t aa = smem_u32(ops + (j % kWgOps) * OPS), bb = aa + ABYTES;
#pragma unroll
      for (int kk = 0; kk < kWgK / 8; ++kk)
        mma_tf32(tmem, make_desc(aa + kk * 256, 128, SBO), make_desc(bb + kk * 256, 128, SBO), idesc,
                 (j > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&obar[j % kWgOps]);
    }
    issued = j;
  }
  // blocks still in flight (only after a failed wait) land before exit
  if (t == 0 && s_fail)
    for (int j = issued + 1; j < nst && j < issued + kWgRaw; ++j)
      (void)mbar_wait_bounded(&rbar[j % kWgRaw], (uint32_t)((j / kWgRaw) & 1));
  // wait for the last issued stage (its commit covers every earlier MMA)
  if (t == 0 && issued >= 0 &&
      !mbar_wait_bounded(&obar[issued % kWgOps], (uint32_t)((issued / kWgOps) & 1)))
    s_fail = 1;
  fence_before();
  __syncthreads();
  fence_after();
  if (!s_fail && issued == nst - 1 && nst > 0) {
    const int qd = warp & 3, half = warp >> 2;
    const int o = qd * 32 + lane;
    double* gW = a.grad + m.poff[l];
    for (int c = half; c < nb / 8; c += 2) {
      uint32_t v[8];
      tmem_ld8_nowait(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(c * 8), v);
      tmem_wait_ld();
      if (o < wo) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int n = c * 8 + u;
          const double x = (double)__uint_as_float(v[u]);
          if (n < wi) atomicAdd(gW + (int64_t)o * wi + n, x);
          else if (n == wi) atomicAdd(gW + (int64_t)wo * wi + o, x);
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (t == 0 && s_fail) atomicExch(m.status, 6);  // BS_TIMEOUT
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// CTAs of a kernel resident per SM, from the device's limits: shared memory
// (dynamic + static + the per-block reservation), threads, registers and the
// tensor-memory columns each CTA allocates.
template <typename K>
cudaError_t prepare(K kern, size_t smem, int threads, uint32_t tmem_cols, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  int dev = 0, sm_smem = 0, reserved = 0, sm_threads = 0, sm_regs = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  int occ = (int)(512 / tmem_cols);
  const size_t per_block = smem + fa.sharedSizeBytes + (size_t)reserved;
  if ((int)(sm_smem / per_block) < occ) occ = (int)(sm_smem / per_block);
  if (sm_threads / threads < occ) occ = sm_threads / threads;
  const int regs = ((fa.numRegs + 7) / 8) * 8 * threads;
  if (regs > 0 && sm_regs / regs < occ) occ = sm_regs / regs;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  *per_sm = occ;
  return cudaSuccess;
}

template <int DIN, int W>
cudaError_t run_tf32(const MlpDev& m, const LossArgs& la, float* ws, const TrainLayout& TL, unsigned char* pack,
                     const unsigned long long* cnt, double* loss_acc, double* grad, cudaStream_t s) {
  const int n_sq = m.n_lin - 2;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  unsigned char* wbwd = pack + (size_t)n_sq * W * W * 4;
  pack_tf32_train_kernel<<<sms, 256, 0, s>>>(m, W, pack, wbwd);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  T32Args ta{};
  ta.m = m;
  ta.la = la;
  ta.ws = ws;
  for (int l = 0; l < 16; ++l) {
    ta.act_off[l] = TL.act_off[l];
    ta.dz_off[l] = TL.dz_off[l];
  }
  ta.wfwd = pack;
  ta.wbwd = wbwd;
  ta.cnt = cnt;
  ta.loss_acc = loss_acc;
  ta.ntiles = (int)((la.N + kT32Pts - 1) / kT32Pts);
  constexpr uint32_t NCOLS = W <= 32 ? 32 : (W <= 64 ? 64 : 128);
  const size_t smem = t32_smem_bytes(W, DIN, m.n_lin);
  int occ_f = 0, occ_b = 0;
  if ((e = prepare(train_tf32_fwd_kernel<DIN, W>, smem, 4 * W, NCOLS, &occ_f)) != cudaSuccess) return e;
  const size_t bsmem = t32_bwd_smem_bytes(W);
  if ((e = prepare(train_tf32_bwd_kernel<DIN, W>, bsmem, 4 * W, NCOLS, &occ_b)) != cudaSuccess) return e;
  const int gf = ta.ntiles < sms * occ_f ? ta.ntiles : sms * occ_f;
  const int gb = ta.ntiles < sms * occ_b ? ta.ntiles : sms * occ_b;
  train_tf32_fwd_kernel<DIN, W><<<gf, 4 * W, smem, s>>>(ta);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  train_tf32_bwd_kernel<DIN, W><<<gb, 4 * W, bsmem, s>>>(ta);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // weight gradient: every layer the same number of CTAs (the rows of a stage
  // cost about the same whatever the layer: the chain of waits, conversion and
  // MMA issue dominates a stage's time, not its bytes)
  WgT32Args wa{};
  wa.m = m;
  wa.X = la.X;
  wa.N = la.N;
  wa.ws = ws;
  for (int l = 0; l < 16; ++l) {
    wa.act_off[l] = TL.act_off[l];
    wa.dz_off[l] = TL.dz_off[l];
  }
  wa.grad = grad;
  const int64_t R = 4 * la.N;
  constexpr uint32_t WG_COLS = W + 16 <= 32 ? 32 : (W + 16 <= 64 ? 64 : (W + 16 <= 128 ? 128 : 256));
  const size_t wsm = wg_smem_bytes<W>();
  int occ_w = 0;
  if ((e = prepare(train_tf32_wgrad_kernel<DIN, W>, wsm, 256, WG_COLS, &occ_w)) != cudaSuccess) return e;
  int c = 0;
  for (int l = 1; l <= m.n_lin; ++l) {
    int k = sms * occ_w / m.n_lin;
    if (k < 1) k = 1;
    const int64_t cr = ((R + k - 1) / k + kWgK - 1) / kWgK * kWgK;
    k = (int)((R + cr - 1) / cr);
    wa.cta0[l] = c;
    wa.crows[l] = cr;
    c += k;
  }
  wa.cta0[m.n_lin + 1] = c;
  train_tf32_wgrad_kernel<DIN, W><<<c, 256, wsm, s>>>(wa);
  return cudaGetLastError();
}

template <int DIN>
cudaError_t run_tf32_w(const MlpDev& m, const LossArgs& la, float* ws, const TrainLayout& TL, unsigned char* pack,
                       const unsigned long long* cnt, double* loss_acc, double* grad, cudaStream_t s) {
  switch (m.widths[1]) {
    case 32:
      return run_tf32<DIN, 32>(m, la, ws, TL, pack, cnt, loss_acc, grad, s);
    case 64:
      return run_tf32<DIN, 64>(m, la, ws, TL, pack, cnt, loss_acc, grad, s);
    case 96:
      return run_tf32<DIN, 96>(m, la, ws, TL, pack, cnt, loss_acc, grad, s);
    case 128:
      return run_tf32<DIN, 128>(m, la, ws, TL, pack, cnt, loss_acc, grad, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool train_tf32_supported(const MlpDev& m) {
  if (m.n_lin < 3 || m.n_lin > 16 || (m.d_in != 2 && m.d_in != 5)) return false;
  const int w = m.widths[1];
  if (w != 32 && w != 64 && w != 96 && w != 128) return false;
  for (int l = 1; l < m.n_lin; ++l)
    if (m.widths[l] != w) return false;
  return m.widths[m.n_lin] == 1;
}

size_t train_tf32_pack_bytes(const MlpDev& m) {
  if (!train_tf32_supported(m)) return 0;
  const size_t w = (size_t)m.widths[1];
  return 2 * (size_t)(m.n_lin - 2) * w * w * 4;
}

cudaError_t launch_train_tf32(const MlpDev& m, const LossArgs& la, float* ws, const TrainLayout& TL,
                              unsigned char* pack, const unsigned long long* cnt, double* loss_acc, double* grad,
                              cudaStream_t s) {
  if (la.N <= 0) return cudaSuccess;
  if (!train_tf32_supported(m) || ((uintptr_t)ws & 15) != 0 || ((uintptr_t)pack & 15) != 0)
    return cudaErrorInvalidValue;
  return m.d_in == 2 ? run_tf32_w<2>(m, la, ws, TL, pack, cnt, loss_acc, grad, s)
                     : run_tf32_w<5>(m, la, ws, TL, pack, cnt, loss_acc, grad, s);
}

}  // namespace bsp
