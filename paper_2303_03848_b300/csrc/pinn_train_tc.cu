// pinn_train_tc.cu -- the weight gradient of the network's square hidden layers
// (Section 3.3 training, the adjoint of Eqs. 11-14) on the tensor cores:
// BF16 operands, FP32 accumulation in tensor memory.
//
// For a hidden layer l with w inputs and w outputs
//   dL/dW_l[o][i] = sum over streams s and points p of dz_s[o][p] * h_s[i][p],
// where dz_s are the adjoints of the layer's four pre-activation streams
// (value, d/dS, d2/dS2, d/dtau) and h_s the streams of its input, rebuilt from
// the stored (t, z_S, z_SS, z_tau) of the layer below:
//   h_0 = t,  h_1 = t' z_S,  h_2 = t' z_SS + t'' z_S^2,  h_3 = t' z_tau,
//   t' = 1 - t^2,  t'' = -2 t t'.
// That is one GEMM D[o][i] = sum_k A[o][k] B[i][k] with K = 4N: A = dz (rows o,
// K = (s, p)), B = h (rows i, K = (s, p)); both are stored point-contiguous, so
// a 64-point slice of a row is a K-major operand chunk.
//
// One CTA of 128 threads owns a 128-row tile of o and a contiguous range of
// (stream, 64-point block) chunks.  Per chunk the threads convert the operands
// to BF16 into one of two shared-memory stages (core-matrix layout) while the
// tensor core works on the other; one thread issues the four K=16 MMAs and
// commits them to the stage's mbarrier.  The FP32 partial sums of each CTA go to
// a buffer that a second kernel adds up in FP64 into the gradient.  Every wait is
// bounded; on expiry the kernel records BS_TIMEOUT and stops.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>

#include "bs_internal.h"
#include "pinn_loss.cuh"
#include "tcgen05.cuh"

namespace bsp {

using namespace tc;

namespace {

constexpr int kChunk = 64;  // points per K chunk

struct WgArgs {
  const float* dz;   // adjoints of layer l: [4][w][N]
  const float* act;  // stored streams of layer l-1: [4][w][N] = (t, z_S, z_SS, z_tau)
  int64_t N;
  int w;
  int nbr;      // rows of B: w, or w + 16 with row w = 1 on the value stream (bias gradient)
  int nb;       // 64-point blocks
  int per_cta;  // chunks per CTA along K
  int vec;      // N % 4 == 0: 16-byte loads
  float* partial;  // [gridDim.y][w][w + 1]
  int* status;
};

// 8 consecutive floats of a row from p = pb on (zero past N).
__device__ __forceinline__ void load8(const float* src, int64_t pb, int64_t N, int vec, float (&v)[8]) {
  if (vec && pb + 8 <= N) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(src));
    const float4 y = __ldg(reinterpret_cast<const float4*>(src + 4));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = pb + e < N ? __ldg(src + e) : 0.0f;
  }
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 q = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&q);
}

__global__ void __launch_bounds__(128) wgrad_tc_kernel(WgArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int w = a.w, t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ot = blockIdx.x;
  constexpr uint32_t a_bytes = 128 * kChunk * 2;
  const int nbr = a.nbr;
  const uint32_t b_bytes = (uint32_t)nbr * kChunk * 2;
  auto stA = [&](int st) { return smem + st * a_bytes; };
  auto stB = [&](int st) { return smem + 2 * a_bytes + st * b_bytes; };
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * a_bytes + 2 * b_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int s_fail;
  const int total = 4 * a.nb;
  const int c0 = blockIdx.y * a.per_cta;
  const int c1 = c0 + a.per_cta < total ? c0 + a.per_cta : total;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  uint32_t ncols = 32;
  while ((int)ncols < nbr) ncols <<= 1;
  if (warp == 0) tmem_alloc(tslot, ncols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc_bf16(nbr);
  const int64_t N = a.N;
  int n = 0;
  for (int c = c0; c < c1; ++c, ++n) {
    const int st = n & 1;
    const int s = c / a.nb;
    const int64_t p0 = (int64_t)(c % a.nb) * kChunk;
    if (n >= 2 && !mbar_wait_bounded(&bar[st], (uint32_t)((n - 2) >> 1) & 1u)) s_fail = 1;  // stage free
    __syncthreads();
    if (s_fail) break;
    // A: 128 rows (o) x 64 points of dz_s, BF16
    for (int it = t; it < 128 * (kChunk / 8); it += 128) {
      const int row = it >> 3, kc = it & 7;
      const int o = ot * 128 + row;
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      if (o < w) {
        const int64_t pb = p0 + kc * 8;
        float v[8];
        load8(a.dz + ((int64_t)s * w + o) * N + pb, pb, N, a.vec, v);
        q = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
      }
      *reinterpret_cast<uint4*>(stA(st) + canon_off(row, kc * 8, kChunk)) = q;
    }
    // B: w rows (i) x 64 points of h_s rebuilt from the stored streams, BF16;
    // then (nbr > w) the bias row (1 on the value stream) and zero rows
    for (int it = t; it < nbr * (kChunk / 8); it += 128) {
      const int i = it >> 3, kc = it & 7;
      const int64_t pb = p0 + kc * 8;
      float v[8];
      if (i >= w) {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (i == w && s == 0 && pb + e < N) ? 1.0f : 0.0f;
      } else {
        float tt[8], zz[8], z1[8];
        load8(a.act + ((int64_t)0 * w + i) * N + pb, pb, N, a.vec, tt);
        if (s != 0) load8(a.act + ((int64_t)(s == 2 ? 2 : (s == 3 ? 3 : 1)) * w + i) * N + pb, pb, N, a.vec, zz);
        if (s == 2) load8(a.act + ((int64_t)1 * w + i) * N + pb, pb, N, a.vec, z1);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float d1 = 1.0f - tt[e] * tt[e];
          if (s == 0) v[e] = tt[e];
          else if (s == 2) v[e] = d1 * zz[e] - 2.0f * tt[e] * d1 * z1[e] * z1[e];
          else v[e] = d1 * zz[e];
        }
      }
      const uint4 q = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
      *reinterpret_cast<uint4*>(stB(st) + canon_off(i, kc * 8, kChunk)) = q;
    }
    fence_proxy_async();  // generic-proxy writes of the stage visible to the tensor core
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      const uint32_t aa = smem_u32(stA(st)), bb = smem_u32(stB(st));
#pragma unroll
      for (int kk = 0; kk < kChunk / 16; ++kk) {
        const uint64_t da = make_desc(aa + kk * 256, 128, (kChunk / 8) * 128);
        const uint64_t db = make_desc(bb + kk * 256, 128, (kChunk / 8) * 128);
        mma_bf16(tmem, da, db, idesc, (n > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&bar[st]);
    }
  }
  // the last commit covers every MMA issued before it
  if (!s_fail && n > 0 && !mbar_wait_bounded(&bar[(n - 1) & 1], (uint32_t)((n - 1) >> 1) & 1u)) s_fail = 1;
  fence_after();
  __syncthreads();
  if (!s_fail && n > 0) {
    const int o = ot * 128 + warp * 32 + lane;
    const int wc = nbr > w ? w + 1 : w;  // columns kept: w, and the bias
    float* dst = a.partial + ((int64_t)blockIdx.y * w + o) * (w + 1);
    for (int cc = 0; cc < wc; cc += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
      if (o < w) {
#pragma unroll
        for (int e = 0; e < 32; ++e)
          if (cc + e < wc) dst[cc + e] = v[e];
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (s_fail && t == 0) atomicExch(a.status, 6);  // BS_TIMEOUT
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// gW[o][i] (i < w) and gb[o] (column w, when the bias row was in the GEMM):
// sums over CTAs of the partial sums; blockIdx.y takes one group of CTAs and
// adds its FP64 sum atomically (the gradient starts at zero).
__global__ void wgrad_sum_kernel(const float* __restrict__ partial, int ny, int w, int with_bias,
                                 double* __restrict__ gW, double* __restrict__ gb) {
  const int64_t wc = (int64_t)w * (w + 1);
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= wc) return;
  const int o = (int)(q / (w + 1)), i = (int)(q % (w + 1));
  if (i == w && !with_bias) return;
  const int y0 = (int)((int64_t)ny * blockIdx.y / gridDim.y), y1 = (int)((int64_t)ny * (blockIdx.y + 1) / gridDim.y);
  float acc = 0.0f;
  for (int y = y0; y < y1; ++y) acc += partial[(int64_t)y * wc + q];
  atomicAdd(i < w ? gW + (int64_t)o * w + i : gb + o, (double)acc);
}

// gb[o] = sum_p dz_0[o][p] for widths without the bias row in the GEMM (w > 240),
// the adjoint rounded to BF16 like the GEMM operand.
__global__ void bias_grad_kernel(const float* __restrict__ dz, int64_t N, double* __restrict__ gb) {
  __shared__ float red[4];
  const int o = blockIdx.x, t = threadIdx.x;
  float acc = 0.0f;
  for (int64_t p = t; p < N; p += blockDim.x) acc += bf16r(dz[(int64_t)o * N + p]);
  for (int s = 16; s >= 1; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
  if ((t & 31) == 0) red[t >> 5] = acc;
  __syncthreads();
  if (t == 0) gb[o] = (double)red[0] + red[1] + red[2] + red[3];
}

// Input layer (d_in -> w): its input streams are the mapped inputs h_0 = x^ and
// the constants h_1 = sc_S e_S, h_3 = sc_tau e_tau (h_2 = 0), so
//   dL/dW_1[o][i] = sum_p dz_0[o][p] x^_i(p) + [i = 0] sc_S sum_p dz_1[o][p]
//                   + [i = 1] sc_tau sum_p dz_3[o][p],   dL/db_1[o] = sum_p dz_0[o][p];
// operands rounded to BF16 like the GEMM operands.  One CTA per (o, chunk).
template <int DIN>
__global__ void grad_input_kernel(MlpDev m, const double* __restrict__ X, int64_t N, const float* __restrict__ dz1,
                                  double* __restrict__ grad, int64_t chunk) {
  __shared__ float red[4][12];
  constexpr int d = DIN;
  const int o = blockIdx.x, t = threadIdx.x, w = m.widths[1];
  const int64_t p0 = (int64_t)blockIdx.y * chunk, p1 = p0 + chunk < N ? p0 + chunk : N;
  float ax[8] = {0, 0, 0, 0, 0, 0, 0, 0}, a0 = 0.0f, a1 = 0.0f, a3 = 0.0f;
  double sc[DIN], lo[DIN];
#pragma unroll
  for (int i = 0; i < d; ++i) {
    sc[i] = 2.0 / (m.hi[i] - m.lo[i]);
    lo[i] = m.lo[i];
  }
  for (int64_t p = p0 + t; p < p1; p += blockDim.x) {
    const float g0 = bf16r(dz1[(0 * (int64_t)w + o) * N + p]);
    a0 += g0;
    a1 += bf16r(dz1[(1 * (int64_t)w + o) * N + p]);
    a3 += bf16r(dz1[(3 * (int64_t)w + o) * N + p]);
#pragma unroll
    for (int i = 0; i < d; ++i) ax[i] += g0 * bf16r((float)(sc[i] * (X[p * d + i] - lo[i]) - 1.0));
  }
  float v[11];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = ax[i];
  v[8] = a0;
  v[9] = a1;
  v[10] = a3;
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    float x = v[k];
    for (int s = 16; s >= 1; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
    if ((t & 31) == 0) red[t >> 5][k] = x;
  }
  __syncthreads();
  if (t < 11 && (t < d || t >= 8)) {
    const double tot = (double)red[0][t] + red[1][t] + red[2][t] + red[3][t];
    double* g = grad + m.poff[1];
    if (t < d) {
      atomicAdd(g + (int64_t)o * d + t, tot);
    } else if (t == 8) {
      atomicAdd(g + (int64_t)w * d + o, tot);
    } else {
      const int i = t == 9 ? 0 : 1;  // d/dS stream feeds input 0 (S), d/dtau stream input 1 (tau)
      const double sc = 2.0 / (m.hi[i] - m.lo[i]);
      atomicAdd(g + (int64_t)o * d + i, (double)bf16r((float)sc) * tot);
    }
  }
}

// Output layer (w -> 1): dL/dW_L[i] = sum_{s,p} dz_s[p] h_s[i][p] with h_s
// rebuilt from the last hidden layer's stored streams; warp i = w is the bias
// (h_0 = 1).  One warp per i, lanes over the points of a chunk.
__global__ void grad_output_kernel(const float* __restrict__ act, const float* __restrict__ seeds, int w, int64_t N,
                                   double* __restrict__ gW, double* __restrict__ gb, int64_t chunk) {
  const int i = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i > w) return;
  const int64_t p0 = (int64_t)blockIdx.y * chunk, p1 = p0 + chunk < N ? p0 + chunk : N;
  float acc = 0.0f;
  for (int64_t p = p0 + lane; p < p1; p += 32) {
    const float g0 = bf16r(seeds[p]);
    if (i == w) {
      acc += g0;
      continue;
    }
    const float g1 = bf16r(seeds[N + p]), g2 = bf16r(seeds[2 * N + p]), g3 = bf16r(seeds[3 * N + p]);
    const float tt = act[(0 * (int64_t)w + i) * N + p], zs = act[(1 * (int64_t)w + i) * N + p];
    const float zss = act[(2 * (int64_t)w + i) * N + p], zt = act[(3 * (int64_t)w + i) * N + p];
    const float d1 = 1.0f - tt * tt;
    acc += g0 * bf16r(tt) + g1 * bf16r(d1 * zs) + g2 * bf16r(d1 * zss - 2.0f * tt * d1 * zs * zs) + g3 * bf16r(d1 * zt);
  }
  for (int s = 16; s >= 1; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
  if (lane == 0) atomicAdd(i < w ? gW + i : gb, (double)acc);
}

// CTAs along K: about two per SM over all o tiles.
void wgrad_grid(int w, int64_t N, int* ot, int* per_cta, int* ny) {
  const int nb = (int)((N + kChunk - 1) / kChunk);
  const int total = 4 * nb;
  *ot = (w + 127) / 128;
  int pc = (int)(((int64_t)total * *ot + 295) / 296);
  if (pc < 1) pc = 1;
  *per_cta = pc;
  *ny = (total + pc - 1) / pc;
}

int wgrad_rows_b(int w) { return w + 16 <= 256 ? w + 16 : w; }

size_t wgrad_smem_bytes(int w) {
  return 2 * (size_t)128 * kChunk * 2 + 2 * (size_t)wgrad_rows_b(w) * kChunk * 2 + 64;
}

// Pack the square layers for training: W_l (rows o, K = i) for the forward and
// W_l^T (rows i, K = o) for the adjoint, BF16 core-matrix layout.
__global__ void pack_train_kernel(MlpDev m, int w, unsigned char* fwd, unsigned char* bwd) {
  const int n_sq = m.n_lin - 2;
  const int64_t per = (int64_t)w * w;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < per * n_sq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int sq = (int)(q / per);
    const int o = (int)((q % per) / w), i = (int)(q % w);
    const __nv_bfloat16 v = __float2bfloat16_rn(m.p32[m.poff[sq + 2] + (int64_t)o * w + i]);
    *reinterpret_cast<__nv_bfloat16*>(fwd + sq * per * 2 + canon_off(o, i, w)) = v;
    *reinterpret_cast<__nv_bfloat16*>(bwd + sq * per * 2 + canon_off(i, o, w)) = v;
  }
}

// ---------------------------------------------------------------------------
// Forward with the four derivative streams on the tensor cores.  A CTA of 128
// threads takes 32 points at a time; row r = 32 s + q of every layer GEMM is
// stream s (warp s) of point q (lane q), so each thread reads its own row of
// the accumulator.  Per hidden layer the value stream's warp forms t = tanh(z)
// and the S-stream's warp publishes z_S through shared memory; then every
// stream forms its input to the next layer:
//   h_0 = t, h_1 = t' z_S, h_2 = t' z_SS + t'' z_S^2, h_3 = t' z_tau,
// stores (t, z_S, z_SS, z_tau) for the adjoint and writes h_s in BF16 as the
// next A operand.  Input layer, output layer and the loss seeds on CUDA cores.
// ---------------------------------------------------------------------------
struct FwdArgs {
  MlpDev m;
  LossArgs la;
  float* act[16];      // act[l], l = 1..n_lin-1: [4][w][N] = (t, z_S, z_SS, z_tau)
  float* seeds;        // dLoss/d(u, u_S, u_SS, u_tau): [4][N]
  const unsigned char* wpack;  // square layers, W_l (rows o, K = i)
  const unsigned long long* cnt;
  double* loss_acc;
};

template <int DIN>
__global__ void __launch_bounds__(128) train_fwd_tc_kernel(FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  const int t = threadIdx.x, s = t >> 5, q = t & 31;
  const int64_t N = a.la.N;
  const uint32_t wbytes = (uint32_t)w * w * 2;
  unsigned char* sW = smem;
  unsigned char* sA = sW + wbytes;
  float* xt = reinterpret_cast<float*>(sA + (size_t)128 * w * 2);  // [2][32][33] tanh of a column chunk
  float* xs = xt + 2 * 32 * 33;                                     // [2][32][33] z_S of a column chunk
  float* sW1 = xs + 2 * 32 * 33;                                    // w x DIN
  float* sB = sW1 + w * DIN;                                        // hidden biases, (n_lin-1) x w
  float* sWo = sB + (m.n_lin - 1) * w;                              // output weights, w
  float* su = sWo + w;                                              // [4][32] output streams
  uint64_t* bar = reinterpret_cast<uint64_t*>(su + 128);            // [0] MMA done, [1] weights landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int s_fail;
  __shared__ double s_acc[3];
  __shared__ float* s_act[16];
  if (t < 16) s_act[t] = a.act[t];

  for (int i = t; i < w * DIN; i += 128) sW1[i] = bf16r(m.p32[m.poff[1] + i]);
  for (int l = 1; l < m.n_lin; ++l)
    for (int o = t; o < w; o += 128) sB[(l - 1) * w + o] = m.p32[m.poff[l] + (int64_t)w * m.widths[l - 1] + o];
  for (int o = t; o < w; o += 128) sWo[o] = bf16r(m.p32[m.poff[m.n_lin] + o]);
  const float bout = m.p32[m.poff[m.n_lin] + w];
  float sc[DIN], of[DIN];
#pragma unroll
  for (int i = 0; i < DIN; ++i) {
    const double g = 2.0 / (m.hi[i] - m.lo[i]);
    sc[i] = (float)g;
    of[i] = (float)(-g * m.lo[i] - 1.0);
  }
  const int64_t ntiles = (N + 31) / 32;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    s_acc[0] = s_acc[1] = s_acc[2] = 0.0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool w_pending = false;
  uint32_t ph_w = 0, ph_mma = 0;
  if (t == 0 && (int64_t)blockIdx.x < ntiles) {
    bulk_load(sW, a.wpack, wbytes, &bar[1]);
    w_pending = true;
  }
  uint32_t ncols = 32;
  while ((int)ncols < w) ncols <<= 1;
  if (s == 0) tmem_alloc(tslot, ncols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc_bf16(w);
  const uint32_t sbo = (uint32_t)(w / 8) * 128;
  const uint32_t trow = tmem + ((uint32_t)(s * 32) << 16);

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * 32 + q;
    const bool valid = p < N;
    const bool last_tile = tile + gridDim.x >= ntiles;
    // input layer on CUDA cores (every stream recomputes the point's z)
    float xh[DIN];
#pragma unroll
    for (int i = 0; i < DIN; ++i) xh[i] = bf16r(fmaf(valid ? (float)a.la.X[p * DIN + i] : 0.0f, sc[i], of[i]));
    {
      float* act1 = s_act[1];
      for (int o0 = 0; o0 < w; o0 += 8) {
        float hv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = o0 + j;
          float z = sB[o];
#pragma unroll
          for (int i = 0; i < DIN; ++i) z = fmaf(sW1[o * DIN + i], xh[i], z);
          const float tt = tanh_fast(z), d1 = 1.0f - tt * tt;
          const float zS = sW1[o * DIN + 0] * sc[0], zT = sW1[o * DIN + 1] * sc[1];
          float h, av;
          if (s == 0) {
            h = tt;
            av = tt;
          } else if (s == 1) {
            h = d1 * zS;
            av = zS;
          } else if (s == 2) {
            h = -2.0f * tt * d1 * zS * zS;
            av = 0.0f;
          } else {
            h = d1 * zT;
            av = zT;
          }
          hv[j] = h;
          if (valid) act1[((int64_t)s * w + o) * N + p] = av;
        }
        *reinterpret_cast<uint4*>(sA + canon_off(t, o0, w)) =
            make_uint4(pack2(hv[0], hv[1]), pack2(hv[2], hv[3]), pack2(hv[4], hv[5]), pack2(hv[6], hv[7]));
      }
    }
    // square layers on the tensor cores
    float dot = 0.0f;
    for (int sq = 0; sq < n_sq; ++sq) {
      const int l = sq + 2;
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
      if (s_fail) break;
      if (t == 0) {
        const uint32_t aa = smem_u32(sA), bb = smem_u32(sW);
        for (int kk = 0; kk < w / 16; ++kk)
          mma_bf16(tmem, make_desc(aa + kk * 256, 128, sbo), make_desc(bb + kk * 256, 128, sbo), idesc,
                   kk > 0 ? 1u : 0u);
        mma_commit(&bar[0]);
      }
      const bool ok = mbar_wait_bounded(&bar[0], ph_mma);
      ph_mma ^= 1u;
      if (!ok) s_fail = 1;
      fence_after();
      if (t == 0 && ok && !(last_tile && sq == n_sq - 1)) {
        const int nxt = sq + 1 < n_sq ? sq + 1 : 0;
        bulk_load(sW, a.wpack + (size_t)nxt * wbytes, wbytes, &bar[1]);
        w_pending = true;
      }
      __syncthreads();
      if (s_fail) break;
      const bool last = sq == n_sq - 1;
      const float* bl = sB + (l - 1) * w;
      float* actl = s_act[l];
      for (int c = 0; c < w; c += 32) {
        const int buf = (c >> 5) & 1;
        float v[32];
        tmem_ld32(trow + (uint32_t)c, v);
        if (s == 0) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            v[j] = tanh_fast(v[j] + bl[c + j]);
            xt[(buf * 32 + q) * 33 + j] = v[j];
          }
        } else if (s == 1) {
#pragma unroll
          for (int j = 0; j < 32; ++j) xs[(buf * 32 + q) * 33 + j] = v[j];
        }
        __syncthreads();
        float hv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float h = v[j];
          if (s != 0) {
            const float tt = xt[(buf * 32 + q) * 33 + j], d1 = 1.0f - tt * tt;
            if (s == 2) {
              const float zS = xs[(buf * 32 + q) * 33 + j];
              h = d1 * v[j] - 2.0f * tt * d1 * zS * zS;
            } else {
              h = d1 * v[j];
            }
          }
          hv[j] = h;
        }
        if (valid) {
#pragma unroll 8
          for (int j = 0; j < 32; ++j) actl[((int64_t)s * w + c + j) * N + p] = v[j];
        }
        if (last) {
#pragma unroll
          for (int j = 0; j < 32; ++j) dot = fmaf(sWo[c + j], bf16r(hv[j]), dot);
        } else {
#pragma unroll
          for (int j = 0; j < 32; j += 8)
            *reinterpret_cast<uint4*>(sA + canon_off(t, c + j, w)) =
                make_uint4(pack2(hv[j], hv[j + 1]), pack2(hv[j + 2], hv[j + 3]), pack2(hv[j + 4], hv[j + 5]),
                           pack2(hv[j + 6], hv[j + 7]));
        }
      }
      fence_before();
    }
    if (s_fail) break;
    // output streams, loss terms and seeds (the value stream's warp)
    su[s * 32 + q] = dot + (s == 0 ? bout : 0.0f);
    __syncthreads();
    if (s == 0 && valid) {
      double xin[8];
#pragma unroll
      for (int i = 0; i < DIN; ++i) xin[i] = a.la.X[p * DIN + i];
      const double out[4] = {(double)su[q], (double)su[32 + q], (double)su[64 + q], (double)su[96 + q]};
      double sqe[3] = {0.0, 0.0, 0.0}, g[4];
      point_loss(a.la, DIN, xin, a.la.kind[p], out, a.cnt, sqe, g);
#pragma unroll
      for (int k = 0; k < 4; ++k) a.seeds[(int64_t)k * N + p] = (float)g[k];
      for (int k = 0; k < 3; ++k)
        if (sqe[k] != 0.0) atomicAdd(&s_acc[k], sqe[k]);
    }
  }
  if (t == 0 && w_pending) (void)mbar_wait_bounded(&bar[1], ph_w);
  fence_before();
  __syncthreads();
  fence_after();
  if (t == 0) {
    atomicAdd(a.loss_acc + 0, s_acc[0]);
    atomicAdd(a.loss_acc + 1, s_acc[1]);
    atomicAdd(a.loss_acc + 2, s_acc[2]);
    if (s_fail) atomicExch(m.status, 6);  // BS_TIMEOUT
  }
  if (s == 0) tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Adjoint on the tensor cores, same tile mapping (row 32 s + q = stream s of
// point q).  From the top hidden layer down: ah_s = W_{l+1}^T dz_{l+1,s} (the
// output layer's is rank one, on CUDA cores; the others one GEMM with the
// packed W^T), then the adjoint of the tanh streams of layer l,
//   t_bar = ah_0 - 2 t' d2_bar - 2 t d1_bar,  d2_bar = ah_2 z_S^2,
//   d1_bar = ah_1 z_S + ah_2 z_SS + ah_3 z_tau - 2 t d2_bar,
//   dz_0 = t' t_bar,  dz_1 = t' ah_1 + 2 t'' z_S ah_2,  dz_2 = t' ah_2,  dz_3 = t' ah_3,
// which needs every stream's ah for the value stream: streams 1..3 form their
// shares (ah_S z_S, ah_SS z_SS, ah_SS z_S^2, ah_tau z_tau) and publish them
// through shared memory, so the value stream's warp reads only t.  dz_l goes to global memory (weight gradient)
// and, in BF16, to the A operand of the next GEMM.
// ---------------------------------------------------------------------------
struct BwdArgs {
  MlpDev m;
  int64_t N;
  const float* act[16];         // act[l], l = 1..n_lin-1
  float* dz[16];                // dz[l], l = 1..n_lin-1 (written)
  const float* seeds;           // dz of the output layer: [4][N]
  const unsigned char* wpackT;  // W_l^T (rows i, K = o), square layers l = 2..n_lin-1
};

__global__ void __launch_bounds__(128) train_bwd_tc_kernel(BwdArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  const int t = threadIdx.x, s = t >> 5, q = t & 31;
  const int64_t N = a.N;
  const uint32_t wbytes = (uint32_t)w * w * 2;
  unsigned char* sW = smem;
  unsigned char* sA = sW + wbytes;
  float* xa = reinterpret_cast<float*>(sA + (size_t)128 * w * 2);  // [2][5][32][33] stream partials
  float* sWo = xa + 2 * 5 * 32 * 33;                                // output weights (BF16-rounded)
  float* sseed = sWo + w;                                           // [4][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sseed + 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int s_fail;
  __shared__ const float* s_act[16];
  __shared__ float* s_dz[16];
  auto XA = [&](int buf, int k, int qq, int j) -> float& { return xa[((buf * 5 + k) * 32 + qq) * 33 + j]; };
  if (t < 16) {
    s_act[t] = a.act[t];
    s_dz[t] = a.dz[t];
  }

  for (int o = t; o < w; o += 128) sWo[o] = bf16r(m.p32[m.poff[m.n_lin] + o]);
  const int64_t ntiles = (N + 31) / 32;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool w_pending = false;
  uint32_t ph_w = 0, ph_mma = 0;
  if (t == 0 && (int64_t)blockIdx.x < ntiles) {
    bulk_load(sW, a.wpackT + (size_t)(n_sq - 1) * wbytes, wbytes, &bar[1]);
    w_pending = true;
  }
  uint32_t ncols = 32;
  while ((int)ncols < w) ncols <<= 1;
  if (s == 0) tmem_alloc(tslot, ncols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc_bf16(w);
  const uint32_t sbo = (uint32_t)(w / 8) * 128;
  const uint32_t trow = tmem + ((uint32_t)(s * 32) << 16);

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * 32 + q;
    const bool valid = p < N;
    const bool last_tile = tile + gridDim.x >= ntiles;
    sseed[s * 32 + q] = valid ? bf16r(a.seeds[(int64_t)s * N + p]) : 0.0f;
    __syncthreads();
    const float seed = sseed[s * 32 + q];
    for (int l = m.n_lin - 1; l >= 1; --l) {
      const float* act = s_act[l];
      float* dzl = s_dz[l];
      const bool top = l == m.n_lin - 1;
      for (int c = 0; c < w; c += 32) {
        const int buf = (c >> 5) & 1;
        float ah[32];
        if (top) {
#pragma unroll
          for (int j = 0; j < 32; ++j) ah[j] = sWo[c + j] * seed;
        } else {
          tmem_ld32(trow + (uint32_t)c, ah);
        }
        // the layer's stored streams at (i, p) this stream needs: t always, z_S
        // for streams 1 and 2, z_SS for stream 2, z_tau for stream 3 (loads
        // issued together); each stream's share of the value stream's adjoint
        // goes to shared memory: 0 ah_S z_S, 1 ah_SS, 2 ah_SS z_S^2,
        // 3 ah_SS z_SS, 4 ah_tau z_tau
        float tv[32], zav[32], zbv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t i = c + j;
          tv[j] = valid ? __ldg(act + (0 * (int64_t)w + i) * N + p) : 0.0f;
          const int ka = s == 3 ? 3 : 1;
          zav[j] = (valid && s >= 1) ? __ldg(act + ((int64_t)ka * w + i) * N + p) : 0.0f;
          zbv[j] = (valid && s == 2) ? __ldg(act + (2 * (int64_t)w + i) * N + p) : 0.0f;
        }
        if (s == 1) {
#pragma unroll
          for (int j = 0; j < 32; ++j) XA(buf, 0, q, j) = ah[j] * zav[j];
        } else if (s == 2) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            XA(buf, 1, q, j) = ah[j];
            XA(buf, 2, q, j) = ah[j] * zav[j] * zav[j];
            XA(buf, 3, q, j) = ah[j] * zbv[j];
          }
        } else if (s == 3) {
#pragma unroll
          for (int j = 0; j < 32; ++j) XA(buf, 4, q, j) = ah[j] * zav[j];
        }
        __syncthreads();
        float dzv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float tt = tv[j];
          const float d1 = 1.0f - tt * tt, d2 = -2.0f * tt * d1;
          float r;
          if (s == 0) {
            const float bar_d2 = XA(buf, 2, q, j);
            float bar_d1 = XA(buf, 0, q, j) + XA(buf, 3, q, j) + XA(buf, 4, q, j);
            float bar_t = ah[j];
            bar_t += -2.0f * d1 * bar_d2;
            bar_d1 += -2.0f * tt * bar_d2;
            bar_t += -2.0f * tt * bar_d1;
            r = d1 * bar_t;
          } else if (s == 1) {
            r = ah[j] * d1 + 2.0f * XA(buf, 1, q, j) * d2 * zav[j];
          } else {
            r = ah[j] * d1;
          }
          dzv[j] = r;
        }
        if (valid) {
#pragma unroll 8
          for (int j = 0; j < 32; ++j) dzl[((int64_t)s * w + c + j) * N + p] = dzv[j];
        }
        if (l >= 2) {
#pragma unroll
          for (int j = 0; j < 32; j += 8)
            *reinterpret_cast<uint4*>(sA + canon_off(t, c + j, w)) =
                make_uint4(pack2(dzv[j], dzv[j + 1]), pack2(dzv[j + 2], dzv[j + 3]), pack2(dzv[j + 4], dzv[j + 5]),
                           pack2(dzv[j + 6], dzv[j + 7]));
        }
      }
      fence_before();
      if (l < 2) break;
      // ah of layer l-1: W_l^T dz_l on the tensor cores
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
      if (s_fail) break;
      if (t == 0) {
        const uint32_t aa = smem_u32(sA), bb = smem_u32(sW);
        for (int kk = 0; kk < w / 16; ++kk)
          mma_bf16(tmem, make_desc(aa + kk * 256, 128, sbo), make_desc(bb + kk * 256, 128, sbo), idesc,
                   kk > 0 ? 1u : 0u);
        mma_commit(&bar[0]);
      }
      const bool ok = mbar_wait_bounded(&bar[0], ph_mma);
      ph_mma ^= 1u;
      if (!ok) s_fail = 1;
      fence_after();
      if (t == 0 && ok && !(last_tile && l == 2)) {
        const int nxt = l - 1 >= 2 ? l - 3 : n_sq - 1;  // W_{l-1}^T, or the next tile's first
        bulk_load(sW, a.wpackT + (size_t)nxt * wbytes, wbytes, &bar[1]);
        w_pending = true;
      }
      __syncthreads();
      if (s_fail) break;
    }
    if (s_fail) break;
  }
  if (t == 0 && w_pending) (void)mbar_wait_bounded(&bar[1], ph_w);
  fence_before();
  __syncthreads();
  fence_after();
  if (s_fail && t == 0) atomicExch(m.status, 6);  // BS_TIMEOUT
  if (s == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

cudaError_t launch_train_bwd_tc(const MlpDev& m, int64_t N, const float* const* act, float* const* dz,
                                const float* seeds, const unsigned char* wpack, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  BwdArgs a{};
  a.m = m;
  a.N = N;
  for (int l = 0; l < 16; ++l) {
    a.act[l] = act[l];
    a.dz[l] = dz[l];
  }
  a.seeds = seeds;
  a.wpackT = wpack + (size_t)n_sq * w * w * 2;
  const size_t smem = (size_t)w * w * 2 + (size_t)128 * w * 2 + sizeof(float) * (10 * 32 * 33 + (size_t)w + 128) + 64;
  cudaError_t e = cudaFuncSetAttribute(train_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(train_bwd_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) !=
      cudaSuccess)
    return e;
  int dev = 0, nsm = 148, sm_smem = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  int per_sm = (int)((size_t)sm_smem / (smem + 2048 + (size_t)reserved));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 3) per_sm = 3;
  const int64_t ntiles = (N + 31) / 32;
  const int64_t grid = ntiles < (int64_t)nsm * per_sm ? ntiles : (int64_t)nsm * per_sm;
  train_bwd_tc_kernel<<<(unsigned)grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_grad_edges_tc(const MlpDev& m, const double* X, int64_t N, const float* dz1, const float* act_top,
                                 const float* seeds, double* grad, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int w = m.widths[1];
  const int64_t chunk = 8192;
  const unsigned nc = (unsigned)((N + chunk - 1) / chunk);
  if (m.d_in == 2)
    grad_input_kernel<2><<<dim3(w, nc), 128, 0, s>>>(m, X, N, dz1, grad, chunk);
  else
    grad_input_kernel<5><<<dim3(w, nc), 128, 0, s>>>(m, X, N, dz1, grad, chunk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double* gL = grad + m.poff[m.n_lin];
  grad_output_kernel<<<dim3((w + 1 + 3) / 4, nc), 128, 0, s>>>(act_top, seeds, w, N, gL, gL + w, chunk);
  return cudaGetLastError();
}

bool train_tc_supported(const MlpDev& m) {
  return wgrad_tc_supported(m) && m.widths[1] <= 128 && (m.d_in == 2 || m.d_in == 5);
}

size_t train_tc_pack_bytes(const MlpDev& m) {
  if (!train_tc_supported(m)) return 0;
  return 2 * (size_t)(m.n_lin - 2) * m.widths[1] * m.widths[1] * 2;
}

cudaError_t launch_train_fwd_tc(const MlpDev& m, const LossArgs& la, float* const* act, float* seeds,
                                unsigned char* wpack, const unsigned long long* cnt, double* loss_acc,
                                cudaStream_t s) {
  if (la.N <= 0) return cudaSuccess;
  if (((uintptr_t)wpack & 15) != 0) return cudaErrorInvalidValue;  // TMA source alignment
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  unsigned char* wpackT = wpack + (size_t)n_sq * w * w * 2;
  pack_train_kernel<<<148, 256, 0, s>>>(m, w, wpack, wpackT);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  FwdArgs a{};
  a.m = m;
  a.la = la;
  for (int l = 0; l < 16; ++l) a.act[l] = act[l];
  a.seeds = seeds;
  a.wpack = wpack;
  a.cnt = cnt;
  a.loss_acc = loss_acc;
  const size_t smem = (size_t)w * w * 2 + (size_t)128 * w * 2 +
                      sizeof(float) * (4 * 32 * 33 + (size_t)w * m.d_in + (size_t)(m.n_lin - 1) * w + w + 128) + 64;
  auto kern = m.d_in == 2 ? train_fwd_tc_kernel<2> : train_fwd_tc_kernel<5>;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  int dev = 0, nsm = 148, sm_smem = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  int per_sm = (int)((size_t)sm_smem / (smem + 2048 + (size_t)reserved));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 3) per_sm = 3;  // tensor memory: <= 128 columns each
  const int64_t ntiles = (la.N + 31) / 32;
  const int64_t grid = ntiles < (int64_t)nsm * per_sm ? ntiles : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}

bool wgrad_tc_supported(const MlpDev& m) {
  if (m.n_lin < 3) return false;
  const int w = m.widths[1];
  if (w < 32 || w > 256 || (w % 32) != 0) return false;
  for (int l = 1; l < m.n_lin; ++l)
    if (m.widths[l] != w) return false;
  return true;
}

size_t wgrad_tc_partial_bytes(const MlpDev& m, int64_t N) {
  if (!wgrad_tc_supported(m) || N <= 0) return 0;
  int ot, pc, ny;
  wgrad_grid(m.widths[1], N, &ot, &pc, &ny);
  return (size_t)ny * m.widths[1] * (m.widths[1] + 1) * sizeof(float);
}

cudaError_t launch_wgrad_tc(const MlpDev& m, int64_t N, const float* dz, const float* act, double* gW, double* gb,
                            float* partial, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int w = m.widths[1];
  int ot, pc, ny;
  wgrad_grid(w, N, &ot, &pc, &ny);
  const int nbr = wgrad_rows_b(w);
  WgArgs a{dz, act, N, w, nbr, (int)((N + kChunk - 1) / kChunk), pc, (N % 4) == 0 ? 1 : 0, partial, m.status};
  const size_t smem = wgrad_smem_bytes(w);
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  wgrad_tc_kernel<<<dim3(ot, ny), 128, smem, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t wc = (int64_t)w * (w + 1);
  const int groups = ny < 8 ? ny : 8;
  wgrad_sum_kernel<<<dim3((unsigned)((wc + 255) / 256), groups), 256, 0, s>>>(partial, ny, w, nbr > w, gW, gb);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (nbr == w) {
    bias_grad_kernel<<<w, 128, 0, s>>>(dz, N, gb);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace bsp
