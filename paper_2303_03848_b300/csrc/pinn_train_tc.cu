// pinn_train_tc.cu -- the loss gradient of one training step (Section 3.3, the
// loss of Eqs. 11-14 and its adjoint) with the network's square hidden layers
// on the tensor cores: BF16 operands, FP32 accumulation in tensor memory.
//
// A tile is 128 collocation points.  Every hidden layer is four GEMMs, one per
// derivative stream s (0 value, 1 d/dS, 2 d2/dS2, 3 d/dtau), each into its own
// tensor-memory accumulator, so lane p of all four holds point p and one
// thread mixes the streams of its point in registers:
//   forward   z_s = W h_s (+ b on the value stream),  t = tanh z_0,
//             h_0 = t, h_1 = t' z_1, h_2 = t' z_2 + t'' z_1^2, h_3 = t' z_3,
//             t' = 1 - t^2, t'' = -2 t t';
//   adjoint   ah_s = W^T dz_s (rank one from the loss seeds at the top), then
//             d2_bar = ah_2 z_1^2, d1_bar = ah_1 z_1 + ah_2 z_2 + ah_3 z_3,
//             t_bar = ah_0 - 2 t' d2_bar - 2 t (d1_bar - 2 t d2_bar),
//             dz_0 = t' t_bar, dz_1 = t' ah_1 + 2 t'' z_1 ah_2, dz_2 = t' ah_2,
//             dz_3 = t' ah_3;
//   gradient  dL/dW[o][i] = sum over streams and points of dz_s[o] h_s[i],
//             dL/db[o] = sum over points of dz_0[o].
//
// Workspace (w the hidden width; a batch runs as chunks of at most 2^19 points,
// NT = the 128-point tiles of one chunk):
//   act[l]  FP16 x 4 [slot][w][128]: (z_0, z_1, z_2, z_3) of hidden layer l >= 2
//           at (neuron, point) of the tile a CTA is working on (z_0 with its
//           bias; one slot per CTA, reused tile after tile: activations live
//           only between a tile's forward and its adjoint, which recomputes
//           t = tanh z_0 so that t' = 1 - t^2 keeps its relative accuracy on
//           saturated neurons); the adjoint reads them with one 8-byte load per
//           neuron, 256 contiguous bytes per warp.  Layer 1 keeps t only (float
//           [slot][w][128]): its z_1 = W_1[o][0] sc_S, z_2 = 0 and
//           z_3 = W_1[o][1] sc_tau are constants per neuron;
//   hb[l]   BF16 [NT][4][128 x w]: h_s of hidden layer l (l < n_lin - 1);
//   dzb[l]  BF16 [NT][4][128 x w]: dz_s of hidden layer l (l >= 2).
// The BF16 blocks keep the GEMM operand layout (rows = points, K = neurons,
// no-swizzle core matrices), written by the forward / adjoint epilogues with
// the same 16-byte stores that fill the next GEMM's operand; the weight
// gradient copies them back with TMA bulk loads and reads them as MN-major
// operands (the neuron index contiguous), so no transpose is ever formed.
// The edge layers' gradients are small GEMMs on the same operands while they
// are in shared memory: the output layer's (w -> 1) in the forward, the top
// layer's h_s against a tile of the BF16 loss seeds; the input layer's
// (d_in -> w) in the adjoint, dz_s of layer 1 against a tile of the mapped
// inputs and constant rows.  The input layer's forward runs on CUDA cores.
// Every wait is bounded; on expiry a kernel records BS_TIMEOUT and stops.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "bs_internal.h"
#include "pinn_loss.cuh"
#include "tcgen05.cuh"

namespace bsp {

using namespace tc;

namespace {

struct TcLayout {
  size_t act[16], hb[16], dzb[16];  // byte offsets by hidden layer l
  size_t partial;                   // float [n_sq][ny][w][w + 1]: weight-gradient partial sums
  size_t pack;                      // BF16 square layers: W_l then W_l^T
  size_t total;
  int nt;     // tiles of 128 points (of one chunk)
  int slots;  // activation slots (CTAs of the forward + adjoint kernel)
  int ny;     // weight-gradient CTAs per square layer
};

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

// Points per pass of the kernels: a larger batch runs as consecutive chunks
// (the gradient and the loss sums accumulate), so the workspace is bounded
// whatever the batch.  BSP_TRAIN_CHUNK overrides the default (rounded up to
// whole 128-point tiles).
int64_t chunk_points() {
  int64_t c = (int64_t)1 << 19;
  if (const char* v = std::getenv("BSP_TRAIN_CHUNK")) {
    const long long x = std::atoll(v);
    if (x > 0) c = (x + 127) / 128 * 128;
  }
  return c;
}

__host__ __device__ constexpr uint32_t tmem_cols_streams(int w) {
  return 4 * w <= 128 ? 128 : (4 * w <= 256 ? 256 : 512);
}

// Columns of one thread's group in the epilogues of the fused kernel: 16 for
// w <= 64 (twice the warps on a tile, each with half the columns), else 32
// (the 128-register cap of 512 threads bounds the warps); threads per CTA:
// 4 lane quadrants x w / cols warps.
__host__ __device__ constexpr int train_cols(int w) { return w <= 64 ? 16 : 32; }
__host__ __device__ constexpr int train_threads(int w) { return 128 * (w / train_cols(w)); }

// Activation slots: one per resident CTA of the forward + adjoint kernel (its
// four accumulators bound the CTAs per SM by the 512 tensor-memory columns),
// each reused tile after tile.
int act_slots(int64_t nt, int w) {
  const int64_t cap = (int64_t)sm_count() * (512 / tmem_cols_streams(w));
  return (int)(nt < cap ? nt : cap);
}

TcLayout tc_layout(const MlpDev& m, int64_t N) {
  TcLayout L{};
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  const int64_t nc = N < chunk_points() ? N : chunk_points();
  const int64_t nt = (nc + 127) / 128;
  L.nt = (int)nt;
  L.slots = act_slots(nt, w);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = (o + bytes + 255) / 256 * 256;
    return r;
  };
  for (int l = 1; l < m.n_lin; ++l) L.act[l] = take((size_t)L.slots * w * 128 * (l == 1 ? 4 : 8));
  for (int l = 1; l < m.n_lin - 1; ++l) L.hb[l] = take((size_t)nt * 4 * 128 * w * 2);
  for (int l = 2; l < m.n_lin; ++l) L.dzb[l] = take((size_t)nt * 4 * 128 * w * 2);
  // one wave of weight-gradient CTAs (one per SM) over all square layers
  int ny = sm_count() / (n_sq > 0 ? n_sq : 1);
  if (ny < 1) ny = 1;
  if ((int64_t)ny > 4 * nt) ny = (int)(4 * nt);
  L.ny = ny;
  L.partial = take((size_t)n_sq * ny * w * (w + 1) * sizeof(float));
  L.pack = take((size_t)2 * n_sq * w * w * 2);
  L.total = o;
  return L;
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 q = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&q);
}

__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

// Pack the square layers: W_l (rows o, K = i) for the forward and W_l^T (rows
// i, K = o) for the adjoint, BF16 core-matrix layout.
// The step's prepass in one launch: pack W and W^T of the square layers,
// zero the gradient (np entries) and count the points of each loss term into
// cnt (zeroed by the caller; kinds 0 interior and 4 data, 1 and 2 boundary, 3 expiry).
__global__ void train_prep_kernel(MlpDev m, int w, unsigned char* fwd, unsigned char* bwd, const int8_t* kind,
                                  int64_t N, unsigned long long* cnt, double* grad, int64_t np, int data_ok) {
  const int n_sq = m.n_lin - 2;
  const int64_t per = (int64_t)w * w;
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = i0; q < per * n_sq; q += stride) {
    const int sq = (int)(q / per);
    const int o = (int)((q % per) / w), i = (int)(q % w);
    const __nv_bfloat16 v = __float2bfloat16_rn(m.p32[m.poff[sq + 2] + (int64_t)o * w + i]);
    *reinterpret_cast<__nv_bfloat16*>(fwd + sq * per * 2 + canon_off(o, i, w)) = v;
    *reinterpret_cast<__nv_bfloat16*>(bwd + sq * per * 2 + canon_off(i, o, w)) = v;
  }
  for (int64_t q = i0; q < np; q += stride) grad[q] = 0.0;
  // points per loss term; a kind outside 0..3, or 4 without values, is counted
  // nowhere and recorded as BS_EINVAL in the network's status word
  unsigned long long c0 = 0, c1 = 0, c2 = 0;
  bool bad = false;
  for (int64_t q = i0; q < N; q += stride) {
    const int k = kind[q];
    if (k == 0 || (k == 4 && data_ok)) ++c0;
    else if (k == 1 || k == 2) ++c1;
    else if (k == 3) ++c2;
    else bad = true;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    c0 += __shfl_down_sync(0xffffffffu, c0, o);
    c1 += __shfl_down_sync(0xffffffffu, c1, o);
    c2 += __shfl_down_sync(0xffffffffu, c2, o);
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (c0) atomicAdd(cnt + 0, c0);
    if (c1) atomicAdd(cnt + 1, c1);
    if (c2) atomicAdd(cnt + 2, c2);
    if (bad && m.status != nullptr) atomicExch(m.status, 1);  // BS_EINVAL
  }
}

// Edge-layer GEMMs: D[j][n] = sum over the tile's 128 points of A[j][p] B[n][p]
// with A a 128 x w operand block read MN-major (rows j = neurons) and B a
// 16-row tile (rows n, K = points) in K-major core matrices: element (n, p) at
//   ((n / 8) * 16 + p / 8) * 128 + (n % 8) * 16 + (p % 8) * 2.
constexpr uint32_t kTileB = 16 * 128 * 2;
__device__ __forceinline__ uint32_t tile_off(int n, int p) {
  return (uint32_t)(((n >> 3) * 16 + (p >> 3)) * 128 + (n & 7) * 16 + (p & 7) * 2);
}

// Issue the 8 K = 16 steps of one edge GEMM (accumulating unless first).
template <int W>
__device__ __forceinline__ void edge_mma(uint32_t d_tmem, uint32_t a_smem, uint32_t b_smem, bool first) {
  const uint32_t idesc = make_idesc_bf16_major(16, true, false);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    mma_bf16(d_tmem, make_desc(a_smem + kk * 2 * (W * 16), W * 16, 128), make_desc(b_smem + kk * 256, 128, 2048),
             idesc, (!first || kk > 0) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Forward and adjoint in one persistent kernel.  A tile's adjoint needs only
// that tile's forward, so the stored FP16 (z_0, z_1, z_2, z_3) are read back
// while they are still in L2 (stored with an evict-last policy) and dropped
// from it after their last use (discard.global.L2: never written back to HBM);
// the BF16 operand blocks for the weight gradient stream out with an
// evict-first policy.  A CTA of train_threads(w) threads: warp v reads
// accumulator lanes 32 (v % 4) .. + 31 (one point per thread) and owns the
// cw = train_cols(w) neurons cw (v / 4) .. + cw - 1 of every layer.  Per
// square layer one thread issues the four stream GEMMs (M = 128 points,
// N = K = w); the weights of the next GEMM (W_l going up, W_l^T coming down)
// are fetched by TMA while the epilogue runs.  Between the two passes the
// output streams, the loss terms and the adjoint seeds are formed per point
// in FP32.
// ---------------------------------------------------------------------------
struct TrainArgs {
  MlpDev m;
  LossArgs la;
  unsigned char* ws;
  TcLayout L;
  const unsigned long long* cnt;
  double* loss_acc;
  double* grad;
};

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void st_hint(uint2* p, uint2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol) : "memory");
}

// Four floats rounded to FP16, packed in order.
__device__ __forceinline__ uint2 pack_half4(float a, float b, float c, float d) {
  __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
  return make_uint2(*reinterpret_cast<uint32_t*>(&lo), *reinterpret_cast<uint32_t*>(&hi));
}

__device__ __forceinline__ float4 unpack_half4(uint2 v) {
  const float2 lo = __half22float2(*reinterpret_cast<__half2*>(&v.x));
  const float2 hi = __half22float2(*reinterpret_cast<__half2*>(&v.y));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

__device__ __forceinline__ void st_hint(float* p, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void st_hint(unsigned char* p, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}

// Drop a 128-byte line from L2 without writing it back (its contents become undefined).
__device__ __forceinline__ void discard_l2(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

template <int DIN, int W>
__global__ void __launch_bounds__(train_threads(W), 1) train_tc_kernel(TrainArgs a) {
  constexpr int CW = train_cols(W), NG = W / CW, NCH = CW / 8;  // group columns, groups, 8-column chunks
  constexpr uint32_t WB = W * W * 2, AB = 128 * W * 2, SBO = (W / 8) * 128;
  constexpr uint32_t NCOLS = tmem_cols_streams(W);
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int n_lin = m.n_lin, n_sq = n_lin - 2;
  unsigned char* sW = smem;                                   // weights of the next GEMM
  unsigned char* sA = smem + WB;                              // [4][AB] A operand: h_s going up, dz_s coming down
  unsigned char* sSeed = sA + 4 * AB;                         // [4] seed tiles (row 0), output-layer GEMM
  unsigned char* sX = sSeed + 4 * kTileB;                     // [3] input tiles, input-layer GEMM
  float* sW1 = reinterpret_cast<float*>(sX + 3 * kTileB);     // W x DIN, BF16-rounded
  float* sB = sW1 + W * DIN;                                  // hidden biases, (n_lin - 1) x W
  float* sWo = sB + (n_lin - 1) * W;                          // output weights, BF16-rounded
  float* sZ1 = sWo + W;                                       // layer 1: z_1 = W_1[o][0] sc_S per neuron
  float* sZ3 = sZ1 + W;                                       // layer 1: z_3 = W_1[o][1] sc_tau per neuron
  float* sred = sZ3 + W;                                      // [NG][4][128] output partial sums
  float* sSd = sred + NG * 4 * 128;                           // [4][128] BF16-rounded seeds of the tile
  uint64_t* bar = reinterpret_cast<uint64_t*>(sSd + 4 * 128);  // [0] GEMMs done, [1] weights landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int s_fail;
  __shared__ double s_acc[3];
  __shared__ float s_icnt[3];  // 1 / points per loss term
  __shared__ unsigned char* s_act[16];
  __shared__ unsigned char* s_hb[16];
  __shared__ unsigned char* s_dzb[16];

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, g = warp >> 2, qd = warp & 3;
  const int pl = qd * 32 + lane, c0 = g * CW;
  const int64_t N = a.la.N;
  const int nt = a.L.nt;
  if (t < 16) {
    s_act[t] = (t >= 1 && t < n_lin) ? a.ws + a.L.act[t] : nullptr;
    s_hb[t] = (t >= 1 && t < n_lin - 1) ? a.ws + a.L.hb[t] : nullptr;
    s_dzb[t] = (t >= 2 && t < n_lin) ? a.ws + a.L.dzb[t] : nullptr;
  }
  // input map x^ = sc x + of to [-1, 1] (in shared memory: it is live in both passes)
  __shared__ float sc[8], of[8];
  if (t < DIN) {
    const double gi = 2.0 / (m.hi[t] - m.lo[t]);
    sc[t] = (float)gi;
    of[t] = (float)(-gi * m.lo[t] - 1.0);
  }
  __syncthreads();
  for (int i = t; i < W * DIN; i += blockDim.x) sW1[i] = bf16r(m.p32[m.poff[1] + i]);
  for (int l = 1; l < n_lin; ++l)
    for (int o = t; o < W; o += blockDim.x) sB[(l - 1) * W + o] = m.p32[m.poff[l] + (int64_t)W * m.widths[l - 1] + o];
  for (int o = t; o < W; o += blockDim.x) {
    sWo[o] = bf16r(m.p32[m.poff[n_lin] + o]);
    sZ1[o] = bf16r(m.p32[m.poff[1] + (int64_t)o * DIN + 0]) * sc[0];
    sZ3[o] = bf16r(m.p32[m.poff[1] + (int64_t)o * DIN + 1]) * sc[1];
  }
  for (int i = t; i < (int)(4 * kTileB / 16); i += blockDim.x) reinterpret_cast<uint4*>(sSeed)[i] = make_uint4(0, 0, 0, 0);
  // input tiles: [0] rows x^_0 .. x^_{d-1} (per tile) and row d = 1 (value
  // stream, bias), [1] row d + 1 = 1 (d/dS stream), [2] row d + 2 = 1 (d/dtau stream)
  for (int i = t; i < (int)(3 * kTileB / 2); i += blockDim.x) {
    const int k = i / (kTileB / 2), e = i % (kTileB / 2);  // tile, element in tile order
    const int n = ((e >> 6) >> 4) * 8 + ((e >> 3) & 7);
    const bool one = (k == 0 && n == DIN) || (k == 1 && n == DIN + 1) || (k == 2 && n == DIN + 2);
    reinterpret_cast<__nv_bfloat16*>(sX)[i] = __float2bfloat16_rn(one ? 1.0f : 0.0f);
  }
  const float bout = m.p32[m.poff[n_lin] + W];
  float dwo = 0.0f, dbo = 0.0f;                  // output layer: row pl of its GEMM, sum of seed_0
  float dw1[8] = {0, 0, 0, 0, 0, 0, 0, 0};       // input layer: row pl of its GEMM
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    s_acc[0] = s_acc[1] = s_acc[2] = 0.0;
    for (int k = 0; k < 3; ++k) s_icnt[k] = a.cnt[k] ? 1.0f / (float)a.cnt[k] : 0.0f;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // weights of GEMM q of a tile: q < n_sq -> W_{q+2} (forward), else W^T of layer
  // 2 n_sq + 1 - q (adjoint, top down)
  const unsigned char* wpack = a.ws + a.L.pack;
  auto wsrc = [&](int q) {
    return q < n_sq ? wpack + (size_t)q * WB : wpack + (size_t)n_sq * WB + (size_t)(2 * n_sq - 1 - q) * WB;
  };
  bool w_pending = false, mma_lost = false;
  uint32_t ph_w = 0, ph_mma = 0;
  if (t == 0 && (int)blockIdx.x < nt) {
    bulk_load(sW, wsrc(0), WB, &bar[1]);
    w_pending = true;
  }
  if (warp == 0) tmem_alloc(tslot, NCOLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tl = tmem + ((uint32_t)(qd * 32) << 16);
  const uint32_t rowoff = (uint32_t)((pl >> 3) * (W / 8) * 128 + (pl & 7) * 16) + (uint32_t)(c0 / 8) * 128;
  const uint64_t keep = policy_evict_last(), stream = policy_evict_first();

  // GEMM q: wait for its weights, the four stream GEMMs of sA with sW, wait for
  // them, then fetch the next weights (if `more`)
  auto gemm = [&](int q, bool more) -> bool {
    if (t == 0 && w_pending) {
      if (mbar_wait_bounded(&bar[1], ph_w)) {
        ph_w ^= 1u;
        w_pending = false;
      } else {
        s_fail = 1;
      }
    }
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (s_fail) return false;
    if (t == 0) {
      const uint32_t aa = smem_u32(sA), bb = smem_u32(sW), idesc = make_idesc_bf16(W);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        for (int kk = 0; kk < W / 16; ++kk)
          mma_bf16(tmem + (uint32_t)(s * W), make_desc(aa + s * AB + kk * 256, 128, SBO),
                   make_desc(bb + kk * 256, 128, SBO), idesc, kk > 0 ? 1u : 0u);
      mma_commit(&bar[0]);
    }
    const bool ok = mbar_wait_bounded(&bar[0], ph_mma);
    ph_mma ^= 1u;
    if (!ok) {
      s_fail = 1;
      mma_lost = true;
    }
    fence_after();
    if (t == 0 && ok && more) {
      bulk_load(sW, wsrc(q + 1 < 2 * n_sq ? q + 1 : 0), WB, &bar[1]);
      w_pending = true;
    }
    __syncthreads();
    return !s_fail;
  };
  // an edge-layer GEMM issued by `issue`, then its 16 result columns of row pl
  auto edge = [&](auto issue, uint32_t (&r)[8]) -> bool {
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (s_fail) return false;
    if (t == 0) {
      issue();
      mma_commit(&bar[0]);
    }
    const bool ok = mbar_wait_bounded(&bar[0], ph_mma);
    ph_mma ^= 1u;
    if (!ok) {
      s_fail = 1;
      mma_lost = true;
    }
    fence_after();
    if (ok && g == 0) {
      tmem_ld8_nowait(tl, r);
      tmem_wait_ld();
    }
    fence_before();
    return ok;
  };

  for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int64_t p = (int64_t)tile * 128 + pl;
    const bool valid = p < N;
    const bool last_tile = tile + (int)gridDim.x >= nt;
    // ---- forward, input layer on CUDA cores: h_0 = t, h_1 = t' z_S, h_2 = t'' z_S^2, h_3 = t' z_tau
    {
      float xh[DIN];
#pragma unroll
      for (int i = 0; i < DIN; ++i) xh[i] = bf16r(fmaf(valid ? (float)a.la.X[p * DIN + i] : 0.0f, sc[i], of[i]));
      float* act = reinterpret_cast<float*>(s_act[1]) + ((size_t)blockIdx.x * W + c0) * 128 + pl;
      unsigned char* hb = s_hb[1] + (size_t)tile * 4 * AB + rowoff;
      unsigned char* sa = sA + rowoff;
#pragma unroll
      for (int k = 0; k < NCH; ++k) {
        float h[4][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = c0 + 8 * k + j;
          float z = sB[o];
#pragma unroll
          for (int i = 0; i < DIN; ++i) z = fmaf(sW1[o * DIN + i], xh[i], z);
          const float tt = tanh_fast(z), d1 = 1.0f - tt * tt;
          const float zS = sZ1[o], zT = sZ3[o];
          h[0][j] = tt;
          h[1][j] = d1 * zS;
          h[2][j] = -2.0f * tt * d1 * zS * zS;
          h[3][j] = d1 * zT;
          st_hint(act + (8 * k + j) * 128, tt, keep);
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint4 q = pack8(h[s]);
          *reinterpret_cast<uint4*>(sa + s * AB + k * 128) = q;
          st_hint(hb + s * AB + k * 128, q, stream);
        }
      }
    }
    // ---- forward, square layers on the tensor cores
    float dot[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int sq = 0; sq < n_sq; ++sq) {
      const int l = sq + 2;
      if (!gemm(sq, true)) break;
      const bool last = l == n_lin - 1;
      const float* bl = sB + (l - 1) * W;
      uint2* act = reinterpret_cast<uint2*>(s_act[l]) + ((size_t)blockIdx.x * W + c0) * 128 + pl;
      unsigned char* hb = last ? nullptr : s_hb[l] + (size_t)tile * 4 * AB + rowoff;
      unsigned char* sa = sA + rowoff;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        uint32_t r[4][8];
#pragma unroll
        for (int s = 0; s < 4; ++s) tmem_ld8_nowait(tl + (uint32_t)(s * W + c0 + 8 * ch), r[s]);
        tmem_wait_ld();
        float h[4][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = c0 + 8 * ch + j;
          const float z1 = __uint_as_float(r[1][j]), z2 = __uint_as_float(r[2][j]), z3 = __uint_as_float(r[3][j]);
          const float z0 = __uint_as_float(r[0][j]) + bl[o];
          const float tt = tanh_fast(z0), d1 = 1.0f - tt * tt;
          h[0][j] = tt;
          h[1][j] = d1 * z1;
          h[2][j] = d1 * z2 - 2.0f * tt * d1 * z1 * z1;
          h[3][j] = d1 * z3;
          st_hint(act + (8 * ch + j) * 128, pack_half4(z0, z1, z2, z3), keep);
          if (last) {
#pragma unroll
            for (int s = 0; s < 4; ++s) dot[s] = fmaf(sWo[o], bf16r(h[s][j]), dot[s]);
          }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint4 q = pack8(h[s]);
          if (!last) st_hint(hb + s * AB + ch * 128, q, stream);
          *reinterpret_cast<uint4*>(sa + s * AB + ch * 128) = q;
        }
      }
      fence_before();
    }
    if (s_fail) break;
    // ---- output streams, loss terms and seeds (one thread per point)
#pragma unroll
    for (int s = 0; s < 4; ++s) sred[(g * 4 + s) * 128 + pl] = dot[s];
    __syncthreads();
    if (g == 0) {  // warps 0-3, one per lane quadrant
      float sd[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sqv = 0.0f;  // a point adds to one loss term
      int term = 0;
      if (valid) {
        float out[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          float u = sred[s * 128 + pl];
#pragma unroll
          for (int gg = 1; gg < NG; ++gg) u += sred[(gg * 4 + s) * 128 + pl];
          out[s] = s == 0 ? u + bout : u;
        }
        float xin[8];
#pragma unroll
        for (int i = 0; i < DIN; ++i) xin[i] = (float)a.la.X[p * DIN + i];
        float gs[4], sqe[3] = {0.0f, 0.0f, 0.0f};
        const int kd = a.la.kind[p];
        const float icnt[3] = {s_icnt[0], s_icnt[1], s_icnt[2]};
        const float yv = (kd == 4 && a.la.y != nullptr) ? (float)a.la.y[p] : 0.0f;
        point_loss_f32(a.la, DIN, xin, kd, yv, out, icnt, sqe, gs);
        term = (kd == 0 || kd == 4) ? 0 : (kd == 3 ? 2 : 1);
        sqv = sqe[0] + sqe[1] + sqe[2];
#pragma unroll
        for (int k = 0; k < 4; ++k) sd[k] = bf16r(gs[k]);
        dbo += sd[0];
      }
      // the warp's squared errors: one FP64 shared atomic per warp and term
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float v = term == k ? sqv : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0f) atomicAdd(&s_acc[k], (double)v);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        sSd[s * 128 + pl] = sd[s];
        *reinterpret_cast<__nv_bfloat16*>(sSeed + s * kTileB + tile_off(0, pl)) = __float2bfloat16_rn(sd[s]);
      }
    }
    // ---- output-layer gradient: sum over streams and points of h_s[i] seed_s
    {
      uint32_t r[8];
      if (!edge(
              [&] {
#pragma unroll
                for (int s = 0; s < 4; ++s)
                  edge_mma<W>(tmem, smem_u32(sA + s * AB), smem_u32(sSeed + s * kTileB), s == 0);
              },
              r))
        break;
      if (g == 0) dwo += __uint_as_float(r[0]);
    }
    // ---- adjoint, top hidden layer down
    float sd[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) sd[s] = sSd[s * 128 + pl];
    for (int l = n_lin - 1; l >= 1; --l) {
      const bool top = l == n_lin - 1;
      const uint2* act = reinterpret_cast<const uint2*>(s_act[l]) + ((size_t)blockIdx.x * W + c0) * 128 + pl;
      const float* act1 = reinterpret_cast<const float*>(s_act[1]) + ((size_t)blockIdx.x * W + c0) * 128 + pl;
      unsigned char* dzb = l >= 2 ? s_dzb[l] + (size_t)tile * 4 * AB + rowoff : nullptr;
      unsigned char* sa = sA + rowoff;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        float4 av[8];
        if (l >= 2) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            av[j] = unpack_half4(act[(8 * ch + j) * 128]);
            av[j].x = tanh_fast(av[j].x);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) av[j] = make_float4(act1[(8 * ch + j) * 128], sZ1[c0 + 8 * ch + j], 0.0f, sZ3[c0 + 8 * ch + j]);
        }
        float ah[4][8];
        if (top) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float wo = sWo[c0 + 8 * ch + j];
#pragma unroll
            for (int s = 0; s < 4; ++s) ah[s][j] = wo * sd[s];
          }
        } else {
          uint32_t r[4][8];
#pragma unroll
          for (int s = 0; s < 4; ++s) tmem_ld8_nowait(tl + (uint32_t)(s * W + c0 + 8 * ch), r[s]);
          tmem_wait_ld();
#pragma unroll
          for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int j = 0; j < 8; ++j) ah[s][j] = __uint_as_float(r[s][j]);
        }
        float dz[4][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float tt = av[j].x, z1 = av[j].y, z2 = av[j].z, z3 = av[j].w;
          const float d1 = 1.0f - tt * tt, d2 = -2.0f * tt * d1;
          const float bd2 = ah[2][j] * z1 * z1;
          float bd1 = ah[1][j] * z1 + ah[2][j] * z2 + ah[3][j] * z3;
          float bt = ah[0][j];
          bt += -2.0f * d1 * bd2;
          bd1 += -2.0f * tt * bd2;
          bt += -2.0f * tt * bd1;
          dz[0][j] = d1 * bt;
          dz[1][j] = ah[1][j] * d1 + 2.0f * ah[2][j] * d2 * z1;
          dz[2][j] = ah[2][j] * d1;
          dz[3][j] = ah[3][j] * d1;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (l < 2 && s == 2) continue;  // the input layer's d2/dS2 stream has a zero input
          const uint4 q = pack8(dz[s]);
          if (l >= 2) st_hint(dzb + s * AB + ch * 128, q, stream);
          *reinterpret_cast<uint4*>(sa + s * AB + ch * 128) = q;
        }
        // the warp's stored activations of these 8 neurons are dead: drop them from L2
        __syncwarp();
        if (l >= 2) {  // 8 neurons x 32 points x 8 bytes: two lines per neuron
          const uint2* wbase =
              reinterpret_cast<const uint2*>(s_act[l]) + ((size_t)blockIdx.x * W + c0 + 8 * ch) * 128 + qd * 32;
          if (lane < 16)
            discard_l2(reinterpret_cast<const unsigned char*>(wbase + (lane >> 1) * 128) + (lane & 1) * 128);
        } else if (lane < 8) {
          discard_l2(reinterpret_cast<const float*>(s_act[1]) + ((size_t)blockIdx.x * W + c0 + 8 * ch + lane) * 128 +
                     qd * 32);
        }
      }
      fence_before();
      if (l >= 2) {
        // ah of layer l - 1: dz_l W_l (B = W_l^T) on the tensor cores
        if (!gemm(n_sq + (n_lin - 1 - l), l > 2 || !last_tile)) break;
        continue;
      }
      // input-layer gradient: dz_0 against (x^, 1), dz_1 and dz_3 against ones
      if (g == 0) {
#pragma unroll
        for (int i = 0; i < DIN; ++i) {
          const float xh = valid ? bf16r(fmaf((float)a.la.X[p * DIN + i], sc[i], of[i])) : 0.0f;
          *reinterpret_cast<__nv_bfloat16*>(sX + tile_off(i, pl)) = __float2bfloat16_rn(xh);
        }
      }
      uint32_t r[8];
      if (!edge(
              [&] {
                const uint32_t aa = smem_u32(sA), xx = smem_u32(sX);
                edge_mma<W>(tmem, aa, xx, true);
                edge_mma<W>(tmem, aa + AB, xx + kTileB, false);
                edge_mma<W>(tmem, aa + 3 * AB, xx + 2 * kTileB, false);
              },
              r))
        break;
      if (g == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) dw1[j] += __uint_as_float(r[j]);
      }
    }
    if (s_fail) break;
  }
  if (t == 0 && w_pending) (void)mbar_wait_bounded(&bar[1], ph_w);
  if (t == 0 && mma_lost) (void)mbar_wait_bounded(&bar[0], ph_mma ^ 1u);  // GEMMs still in flight
  fence_before();
  __syncthreads();
  fence_after();
  if (g == 0 && !s_fail) {
    double* gL = a.grad + m.poff[n_lin];
    atomicAdd(gL + W, (double)dbo);
    if (pl < W) {
      atomicAdd(gL + pl, (double)dwo);
      // dL/dW_1[o][i] = sum dz_0 x^_i (+ sc_S sum dz_1 for i = 0, + sc_tau sum dz_3 for
      // i = 1: the constant streams of the mapped inputs), dL/db_1[o] = sum dz_0
      double* g1 = a.grad + m.poff[1];
      const double sS = (double)bf16r(sc[0]), sT = (double)bf16r(sc[1]);
#pragma unroll
      for (int i = 0; i < DIN; ++i) {
        double v = (double)dw1[i];
        if (i == 0) v += sS * (double)dw1[DIN + 1];
        if (i == 1) v += sT * (double)dw1[DIN + 2];
        atomicAdd(g1 + (int64_t)pl * DIN + i, v);
      }
      atomicAdd(g1 + (int64_t)W * DIN + pl, (double)dw1[DIN]);
    }
  }
  if (t == 0) {
    atomicAdd(a.loss_acc + 0, s_acc[0]);
    atomicAdd(a.loss_acc + 1, s_acc[1]);
    atomicAdd(a.loss_acc + 2, s_acc[2]);
    if (s_fail) atomicExch(m.status, 6);  // BS_TIMEOUT
  }
  if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ---------------------------------------------------------------------------
// Weight gradient of the square layers: D[o][i] = sum_k A[o][k] B[i][k] over
// k = (tile, stream, point), A = dz_s (the dzb blocks of layer l), B = h_s (the
// hb blocks of layer l - 1), both MN-major; M = 128 rows of o (rows o >= w are
// ignored), N = w, K = 16 points per MMA.  The bias gradient is a second MMA
// on the value-stream blocks with a constant all-ones B (N = 16) into columns
// w .. w + 15.  One thread streams the CTA's range of blocks through S shared
// memory stages with TMA bulk copies and issues the MMAs; the FP32 partial
// sums go to a buffer that wgrad_sum_kernel adds up in FP64.
// ---------------------------------------------------------------------------
struct WgArgs {
  unsigned char* ws;
  TcLayout L;
  int* status;
};

template <int W>
struct WgShape {
  static constexpr uint32_t AB = 128 * W * 2;
  static constexpr uint32_t PAD = 2048;  // rows o >= w of the last K step read up to 2 KB past a block
  static constexpr uint32_t SA = AB + PAD, ST = SA + AB;
  static constexpr int S = (W == 128) ? 3 : 4;
  static constexpr uint32_t NCOLS = W + 16 <= 64 ? 64 : (W + 16 <= 128 ? 128 : 256);
};

template <int W>
__global__ void __launch_bounds__(128) train_wgrad_tc_kernel(WgArgs a) {
  using G = WgShape<W>;
  constexpr int S = G::S;
  constexpr uint32_t KG = W * 16;  // bytes between 8-point groups of a block
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* ones = smem + S * G::ST;  // 16 x 16 BF16 ones
  uint64_t* full = reinterpret_cast<uint64_t*>(ones + 512);
  uint64_t* empty = full + S;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + S);
  __shared__ int s_fail, s_bias;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int sq = blockIdx.y, l = sq + 2;
  const int total = 4 * a.L.nt;
  const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
  const int c0 = (int)blockIdx.x * per;
  const int cnt = c0 < total ? (c0 + per < total ? per : total - c0) : 0;
  const unsigned char* A = a.ws + a.L.dzb[l] + (size_t)c0 * G::AB;
  const unsigned char* B = a.ws + a.L.hb[l - 1] + (size_t)c0 * G::AB;
  for (int i = t; i < 128; i += 128) reinterpret_cast<uint32_t*>(ones)[i] = 0x3F803F80u;
  if (t == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    s_fail = 0;
    s_bias = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, G::NCOLS);
  fence_proxy_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  if (t == 0 && cnt > 0) {
    const uint32_t idm = make_idesc_bf16_major(W, true, true);
    const uint32_t idb = make_idesc_bf16_major(16, true, false);
    const uint64_t dones = make_desc(smem_u32(ones), 128, 256);
    auto load = [&](int n) {
      unsigned char* st = smem + (n % S) * G::ST;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&full[n % S])),
                   "r"(2 * G::AB)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(st)),
                   "l"(A + (size_t)n * G::AB), "r"(G::AB), "r"(smem_u32(&full[n % S]))
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(st + G::SA)),
                   "l"(B + (size_t)n * G::AB), "r"(G::AB), "r"(smem_u32(&full[n % S]))
                   : "memory");
    };
    const int pre = cnt < S ? cnt : S;
    for (int n = 0; n < pre; ++n) load(n);
    int loaded = pre, landed = 0, committed = 0;
    bool fail = false, bias = false;
    for (int n = 0; n < cnt; ++n) {
      const int st = n % S;
      if (!mbar_wait_bounded(&full[st], (uint32_t)(n / S) & 1u)) {
        fail = true;
        break;
      }
      landed = n + 1;
      fence_after();
      const bool value = ((c0 + n) & 3) == 0;
      const uint32_t aa = smem_u32(smem + st * G::ST), bb = aa + G::SA;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const uint64_t da = make_desc(aa + kk * 2 * KG, KG, 128);
        mma_bf16(tmem, da, make_desc(bb + kk * 2 * KG, KG, 128), idm, (n > 0 || kk > 0) ? 1u : 0u);
        if (value) mma_bf16(tmem + W, da, dones, idb, (bias || kk > 0) ? 1u : 0u);
      }
      if (value) bias = true;
      mma_commit(&empty[st]);
      committed = n + 1;
      const int pm = n - 1;  // refill the previous chunk's stage
      if (pm >= 0 && pm + S < cnt) {
        if (!mbar_wait_bounded(&empty[pm % S], (uint32_t)(pm / S) & 1u)) {
          fail = true;
          break;
        }
        load(pm + S);
        loaded = pm + S + 1;
      }
    }
    // the last commit covers every MMA issued before it
    if (committed > 0 &&
        !mbar_wait_bounded(&empty[(committed - 1) % S], (uint32_t)((committed - 1) / S) & 1u))
      fail = true;
    // after a failure: copies still in flight land before the stages are released
    for (int n = landed; fail && n < loaded; ++n) (void)mbar_wait_bounded(&full[n % S], (uint32_t)(n / S) & 1u);
    s_fail = fail ? 1 : 0;
    s_bias = bias ? 1 : 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const int o = warp * 32 + lane;  // accumulator lane = row o
  float* dst = reinterpret_cast<float*>(a.ws + a.L.partial) +
               ((size_t)(sq * (int)gridDim.x + (int)blockIdx.x) * W + (o < W ? o : 0)) * (W + 1);
  const bool have = cnt > 0 && !s_fail;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
  for (int cc = 0; cc < W; cc += 16) {
    uint32_t r[16];
    tmem_ld16_nowait(tl + (uint32_t)cc, r);
    tmem_wait_ld();
    if (o < W) {
#pragma unroll
      for (int e = 0; e < 16; ++e) dst[cc + e] = have ? __uint_as_float(r[e]) : 0.0f;
    }
  }
  {
    uint32_t r[8];
    tmem_ld8_nowait(tl + (uint32_t)W, r);
    tmem_wait_ld();
    if (o < W) dst[W] = (have && s_bias) ? __uint_as_float(r[0]) : 0.0f;
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (s_fail && t == 0) atomicExch(a.status, 6);  // BS_TIMEOUT
  if (warp == 0) tmem_dealloc(tmem, G::NCOLS);
}

// gW[o][i] and gb[o] of square layer blockIdx.z + 2: sums over the layer's
// CTAs of the partial sums; blockIdx.y takes one group of CTAs and adds its
// sum atomically in FP64 (the gradient starts at zero).
// With loss3 set (the batch's last chunk), block (0, 0, 0) also writes the
// loss terms: each sum over its points divided by their count.
__global__ void wgrad_sum_kernel(MlpDev m, const float* __restrict__ partial, int ny, double* __restrict__ grad,
                                 const double* loss_acc, const unsigned long long* cnt, double* loss3) {
  if (loss3 != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) loss3[k] = cnt[k] ? loss_acc[k] / (double)cnt[k] : 0.0;
  }
  const int w = m.widths[1], sq = blockIdx.z;
  const int64_t wc = (int64_t)w * (w + 1);
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= wc) return;
  const int o = (int)(q / (w + 1)), i = (int)(q % (w + 1));
  const int y0 = (int)((int64_t)ny * blockIdx.y / gridDim.y), y1 = (int)((int64_t)ny * (blockIdx.y + 1) / gridDim.y);
  float acc = 0.0f;
  for (int y = y0; y < y1; ++y) acc += partial[((int64_t)sq * ny + y) * wc + q];
  double* gW = grad + m.poff[sq + 2];
  atomicAdd(i < w ? gW + (int64_t)o * w + i : gW + (int64_t)w * w + o, (double)acc);
}

// CTAs of a kernel that fit on one SM at once (shared memory, threads,
// registers, tensor-memory columns); the persistent grids are sized with it.
template <typename K>
int resident_per_sm(K kern, size_t smem, int threads, uint32_t tmem_cols) {
  int dev = 0, sm_smem = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, kern);
  int per = (int)((size_t)sm_smem / (smem + fa.sharedSizeBytes + (size_t)reserved));
  if (per > 2048 / threads) per = 2048 / threads;
  if (fa.numRegs > 0 && per > 65536 / (((fa.numRegs + 7) / 8) * 8 * threads))
    per = 65536 / (((fa.numRegs + 7) / 8) * 8 * threads);
  if (per > (int)(512 / tmem_cols)) per = (int)(512 / tmem_cols);
  return per < 1 ? 1 : per;
}

template <int DIN, int W>
cudaError_t run_train_tc(const MlpDev& m, const LossArgs& la, unsigned char* ws, const TcLayout& L,
                         const unsigned long long* cnt, double* loss_acc, double* grad, double* loss3,
                         cudaStream_t s) {
  constexpr uint32_t WB = W * W * 2, AB = 128 * W * 2;
  const int n_lin = m.n_lin, n_sq = n_lin - 2, nsm = sm_count();
  cudaError_t e;
  {
    TrainArgs a{m, la, ws, L, cnt, loss_acc, grad};
    const size_t smem = WB + 4 * AB + 7 * kTileB +
                        sizeof(float) * ((size_t)W * DIN + (size_t)(n_lin - 1) * W + 3 * W +
                                         (size_t)(W / train_cols(W)) * 4 * 128 +
                                         4 * 128) +
                        64;
    auto kern = train_tc_kernel<DIN, W>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    const int64_t cap = (int64_t)nsm * resident_per_sm(kern, smem, train_threads(W), tmem_cols_streams(W));
    int64_t grid = L.nt < cap ? L.nt : cap;
    if (grid > L.slots) grid = L.slots;
    kern<<<(unsigned)grid, train_threads(W), smem, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    // all of the opt-in shared memory: a descriptor read past the stages stays inside it
    auto kern = train_wgrad_tc_kernel<W>;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    using G = WgShape<W>;
    const size_t need = (size_t)G::S * G::ST + 512 + 2 * G::S * 8 + 16;
    const size_t avail = (size_t)optin - fa.sharedSizeBytes;
    if (need > avail) return cudaErrorInvalidValue;
    const size_t smem = avail;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    kern<<<dim3((unsigned)L.ny, (unsigned)n_sq), 128, smem, s>>>(WgArgs{ws, L, m.status});
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t wc = (int64_t)W * (W + 1);
    const int groups = L.ny < 8 ? L.ny : 8;
    wgrad_sum_kernel<<<dim3((unsigned)((wc + 255) / 256), (unsigned)groups, (unsigned)n_sq), 256, 0, s>>>(
        m, reinterpret_cast<const float*>(ws + L.partial), L.ny, grad, loss_acc, cnt, loss3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int DIN>
cudaError_t run_train_tc_w(const MlpDev& m, const LossArgs& la, unsigned char* ws, const TcLayout& L,
                           const unsigned long long* cnt, double* loss_acc, double* grad, double* loss3,
                           cudaStream_t s) {
  switch (m.widths[1]) {
    case 32:
      return run_train_tc<DIN, 32>(m, la, ws, L, cnt, loss_acc, grad, loss3, s);
    case 64:
      return run_train_tc<DIN, 64>(m, la, ws, L, cnt, loss_acc, grad, loss3, s);
    case 96:
      return run_train_tc<DIN, 96>(m, la, ws, L, cnt, loss_acc, grad, loss3, s);
    case 128:
      return run_train_tc<DIN, 128>(m, la, ws, L, cnt, loss_acc, grad, loss3, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool train_tc_supported(const MlpDev& m) {
  if (m.n_lin < 3 || m.n_lin > 16 || (m.d_in != 2 && m.d_in != 5)) return false;
  const int w = m.widths[1];
  if (w != 32 && w != 64 && w != 96 && w != 128) return false;
  for (int l = 1; l < m.n_lin; ++l)
    if (m.widths[l] != w) return false;
  return m.widths[m.n_lin] == 1;
}

size_t train_tc_workspace_bytes(const MlpDev& m, int64_t N) {
  if (!train_tc_supported(m) || N <= 0) return 0;
  return tc_layout(m, N).total;
}

cudaError_t launch_train_tc(const MlpDev& m, const LossArgs& la, unsigned char* ws, unsigned long long* cnt,
                            double* loss_acc, double* grad, double* loss3, cudaStream_t s) {
  if (la.N <= 0) return cudaSuccess;
  if (!train_tc_supported(m) || ((uintptr_t)ws & 255) != 0) return cudaErrorInvalidValue;
  const TcLayout L = tc_layout(m, la.N);
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  int64_t np = 0;
  for (int l = 1; l <= m.n_lin; ++l) np += (int64_t)m.widths[l] * m.widths[l - 1] + m.widths[l];
  unsigned char* wpack = ws + L.pack;
  train_prep_kernel<<<sm_count(), 256, 0, s>>>(m, w, wpack, wpack + (size_t)n_sq * w * w * 2, la.kind, la.N, cnt,
                                               grad, np, la.y != nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // consecutive chunks of the batch; the loss terms are means over the whole
  // batch (cnt), the gradient and loss sums accumulate
  const int64_t chunk = chunk_points();
  for (int64_t off = 0; off < la.N; off += chunk) {
    LossArgs lc = la;
    lc.X = la.X + off * m.d_in;
    lc.kind = la.kind + off;
    lc.y = la.y != nullptr ? la.y + off : nullptr;
    lc.N = la.N - off < chunk ? la.N - off : chunk;
    TcLayout Lc = L;
    Lc.nt = (int)((lc.N + 127) / 128);
    double* l3 = off + chunk >= la.N ? loss3 : nullptr;  // the last chunk finishes the loss terms
    e = m.d_in == 2 ? run_train_tc_w<2>(m, lc, ws, Lc, cnt, loss_acc, grad, l3, s)
                    : run_train_tc_w<5>(m, lc, ws, Lc, cnt, loss_acc, grad, l3, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bsp
