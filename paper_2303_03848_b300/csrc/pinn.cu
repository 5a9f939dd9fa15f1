// pinn.cu -- the physics-informed network of Section 3.3: evaluation with
// input derivatives, the residual/boundary/expiry loss (Eqs. 11-14), its
// hand-written adjoint (the paper uses automatic differentiation) and Adam.
//
// Network: h_0 = affine map of the inputs to [-1, 1]; h_l = tanh(W_l h_{l-1} + b_l)
// for hidden layers; u = W_L h_{L-1} + b_L.  Derivative streams in S and tau
// are carried forward through every layer:
//   z' = W h',  h' = t' z',  h'' = t' z'' + t'' (z')^2,  t' = 1 - t^2,  t'' = -2 t t'.
//
// This translation unit holds the SIMT paths: FP64 and FP32 arithmetic, and
// TF32 / BF16 operand rounding with FP32 accumulation for networks whose
// hidden layers are not all w x w.  TF32 / BF16 evaluation of w x w hidden
// layers runs on the tensor cores (pinn_tc.cu).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>

#include "bs_internal.h"
#include "pinn_loss.cuh"

namespace bsp {

// ---------------------------------------------------------------------------
// Operand rounding for the reduced-precision modes (RND: 0 none, 1 TF32, 2 BF16).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <int RND>
__device__ __forceinline__ float rop(float x) {
  if (RND == 1) return round_tf32(x);
  if (RND == 2) return round_bf16(x);
  return x;
}
template <int RND>
__device__ __forceinline__ double rop(double x) {
  return x;
}

template <typename Tp>
__device__ __forceinline__ Tp tanh_t(Tp x);
template <>
__device__ __forceinline__ double tanh_t<double>(double x) {
  return tanh(x);
}
template <>
__device__ __forceinline__ float tanh_t<float>(float x) {
  return tanhf(x);
}

template <typename Tp>
__device__ __forceinline__ const Tp* params_of(const MlpDev& m);
template <>
__device__ __forceinline__ const double* params_of<double>(const MlpDev& m) {
  return m.p64;
}
template <>
__device__ __forceinline__ const float* params_of<float>(const MlpDev& m) {
  return m.p32;
}

// Input map of one point: value and derivative streams of the first layer's input.
template <typename Tp>
__device__ __forceinline__ void input_streams(const MlpDev& m, const double* x, Tp* h, Tp* hS, Tp* hSS, Tp* hT,
                                              int stride) {
  for (int i = 0; i < m.d_in; ++i) {
    const double sc = 2.0 / (m.hi[i] - m.lo[i]);
    h[i * stride] = (Tp)(sc * (x[i] - m.lo[i]) - 1.0);
    if (hS) {
      hS[i * stride] = (Tp)((i == 0) ? sc : 0.0);
      hSS[i * stride] = (Tp)0;
      hT[i * stride] = (Tp)((i == 1) ? sc : 0.0);
    }
  }
}

// ---------------------------------------------------------------------------
// Evaluation on CUDA cores as one tiled GEMM per layer.  A CTA of 256 threads
// takes a tile of 64 rows: 64 points, or 16 points x 4 derivative streams with
// the streams of a point on 4 adjacent rows, so that the thread that holds a
// point's four rows forms h_S, h_SS, h_tau of its neurons in registers.  The
// tile's activations live in shared memory neuron-major ([w][64 + 4]: the 4
// rows a thread needs at one k are one vector load); a layer's weights are
// staged transposed ([k][o], 32 values of k at a time, zero-padded to 16 RN
// outputs, rows padded by 4 against bank conflicts), read from global memory
// along k so that a warp's loads are contiguous.  Thread (row group rg, column group cg) accumulates the 4 x RN
// block rows 4 rg .. + 3, outputs RN cg .. + RN - 1 over k -- per k one vector
// load of its rows' activations and RN / 4 (FP32) or RN / 2 (FP64) vector
// loads of weights for 4 RN FMAs -- then writes tanh of the block back over
// the tile once every thread has read it.  The output layer (w -> 1) is a dot
// product per row, four threads a row.
// ---------------------------------------------------------------------------
constexpr int kEvRows = 64;
constexpr int kEvRS = kEvRows + 4;  // row stride of the neuron-major tile (16-byte aligned)

// Offset of neuron k's row in a neuron-major tile: every group of 8 rows is
// shifted by 4 more elements, so that the 16 column groups of a warp, whose
// blocks start 8 k apart, store their rows into different banks.
__host__ __device__ constexpr int hrow(int k) { return k * kEvRS + (k >> 3) * 4; }
__host__ __device__ constexpr int hrows_size(int n) { return hrow(n); }
constexpr int kEvThreads = 256;
constexpr int kEvKC = 32;
constexpr int kEvIn = 8;  // input streams per row (d_in <= 8)

template <typename Tp, int RN>
__device__ __forceinline__ void load_vec(const Tp* __restrict__ p, Tp (&b)[RN]) {
  if constexpr (sizeof(Tp) == 4 && RN % 4 == 0) {
#pragma unroll
    for (int q = 0; q < RN; q += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + q);
      b[q] = v.x;
      b[q + 1] = v.y;
      b[q + 2] = v.z;
      b[q + 3] = v.w;
    }
  } else if constexpr (sizeof(Tp) == 8 && RN % 2 == 0) {
#pragma unroll
    for (int q = 0; q < RN; q += 2) {
      const double2 v = *reinterpret_cast<const double2*>(p + q);
      b[q] = v.x;
      b[q + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < RN; ++q) b[q] = p[q];
  }
}

template <typename Tp>
__device__ __forceinline__ void store4(Tp* p, Tp a, Tp b, Tp c, Tp d) {
  if constexpr (sizeof(Tp) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
    *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
  }
}

template <typename Tp>
constexpr size_t eval_smem_bytes(int RN) {
  return sizeof(Tp) * ((size_t)hrows_size(16 * RN) + (size_t)kEvKC * (16 * RN + 4) + (size_t)hrows_size(kEvIn));
}

template <typename Tp, int RND, int NS, int RN>
__global__ void __launch_bounds__(kEvThreads) mlp_eval_kernel(MlpDev m, const double* __restrict__ X, int64_t N,
                                                              double* __restrict__ u, double* __restrict__ derivs) {
  constexpr int WPAD = 16 * RN, WTS = WPAD + 4, PPT = kEvRows / NS;
  extern __shared__ __align__(16) unsigned char smraw[];
  Tp* H = reinterpret_cast<Tp*>(smraw);  // [WPAD][kEvRS] activations of the tile, neuron-major
  Tp* Wt = H + hrows_size(WPAD);             // [kEvKC][WTS] staged weights, W_l[o][kc + k] at [k][o]
  Tp* Hin = Wt + kEvKC * WTS;            // [kEvIn][kEvRS] input streams
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
  const int r0 = rg * 4, c0 = cg * RN;
  const int64_t p0 = (int64_t)blockIdx.x * PPT;
  // input streams: the value x^ = affine map to [-1, 1], d/dS = (sc_0, 0, ...),
  // d2/dS2 = 0, d/dtau = (0, sc_1, 0, ...)
  for (int i = tid; i < kEvIn * kEvRows; i += kEvThreads) {
    const int k = i / kEvRows, r = i % kEvRows;
    const int pr = r / NS, st = r % NS;
    const int64_t p = p0 + pr;
    Tp v = (Tp)0;
    if (k < m.d_in && p < N) {
      const double sc = 2.0 / (m.hi[k] - m.lo[k]);
      if (st == 0) v = rop<RND>((Tp)(sc * (X[p * m.d_in + k] - m.lo[k]) - 1.0));
      else if (st == 1) v = k == 0 ? (Tp)sc : (Tp)0;
      else if (st == 3) v = k == 1 ? (Tp)sc : (Tp)0;
    }
    Hin[hrow(k) + r] = v;
  }
  const Tp* prm = params_of<Tp>(m);
  for (int l = 1; l < m.n_lin; ++l) {  // hidden layers
    const int wi = m.widths[l - 1], wo = m.widths[l];
    const Tp* Wl = prm + m.poff[l];
    const Tp* bl = Wl + (int64_t)wo * wi;
    const Tp* Hs = l == 1 ? Hin : H;
    Tp acc[4][RN];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < RN; ++q) acc[r][q] = (Tp)0;
    for (int kc = 0; kc < wi; kc += kEvKC) {
      const int kn = wi - kc < kEvKC ? wi - kc : kEvKC;
      __syncthreads();  // the previous chunk is consumed (and, at kc = 0, the tile written)
      for (int i = tid; i < kEvKC * WPAD; i += kEvThreads) {
        const int o = i / kEvKC, k = i % kEvKC;
        Wt[k * WTS + o] = (k < kn && o < wo) ? rop<RND>(Wl[(int64_t)o * wi + kc + k]) : (Tp)0;
      }
      __syncthreads();
      for (int k = 0; k < kn; ++k) {
        Tp a[4], b[RN];
        load_vec<Tp, 4>(Hs + hrow(kc + k) + r0, a);
        load_vec<Tp, RN>(Wt + k * WTS + c0, b);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < RN; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
      }
    }
    __syncthreads();  // every thread has read the tile before it is overwritten
#pragma unroll
    for (int q = 0; q < RN; ++q) {
      const int o = c0 + q;
      const bool ok = o < wo;
      const Tp bias = ok ? bl[o] : (Tp)0;
      Tp h[4];
      if constexpr (NS == 1) {
#pragma unroll
        for (int r = 0; r < 4; ++r) h[r] = ok ? rop<RND>(tanh_t<Tp>(acc[r][q] + bias)) : (Tp)0;
      } else {
        // rows r0 .. r0 + 3: the value and the S, SS, tau streams of one point
        const Tp z = acc[0][q] + bias, zS = acc[1][q], zSS = acc[2][q], zT = acc[3][q];
        const Tp t = tanh_t<Tp>(z);
        const Tp d1 = (Tp)1 - t * t;
        h[0] = ok ? rop<RND>(t) : (Tp)0;
        h[1] = ok ? rop<RND>(d1 * zS) : (Tp)0;
        h[2] = ok ? rop<RND>(d1 * zSS - (Tp)2 * t * d1 * zS * zS) : (Tp)0;
        h[3] = ok ? rop<RND>(d1 * zT) : (Tp)0;
      }
      store4<Tp>(H + hrow(o) + r0, h[0], h[1], h[2], h[3]);
    }
  }
  __syncthreads();
  // output layer (w -> 1, linear): four threads per row, a strided quarter each
  {
    const int wi = m.widths[m.n_lin - 1];
    const Tp* Wo = prm + m.poff[m.n_lin];
    const Tp* Hs = m.n_lin == 1 ? Hin : H;
    const int row = tid >> 2, part = tid & 3;
    Tp z = (Tp)0;
    for (int k = part; k < wi; k += 4) z = fma(rop<RND>(Wo[k]), Hs[hrow(k) + row], z);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    const int64_t p = p0 + row / NS;
    const int st = row % NS;
    if (part == 0 && p < N) {
      if (st == 0) {
        u[p] = (double)(z + Wo[wi]);
      } else if (derivs != nullptr) {
        derivs[3 * p + st - 1] = (double)z;
      }
    }
  }
}

template <typename Tp, int RND, int NS, int RN>
static cudaError_t eval_launch_rn(const MlpDev& m, const double* X, int64_t N, double* u, double* derivs,
                                  cudaStream_t s) {
  const size_t smem = eval_smem_bytes<Tp>(RN);
  cudaError_t e = cudaFuncSetAttribute(mlp_eval_kernel<Tp, RND, NS, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  constexpr int PPT = kEvRows / NS;
  const int64_t blocks = (N + PPT - 1) / PPT;
  mlp_eval_kernel<Tp, RND, NS, RN><<<(unsigned)blocks, kEvThreads, smem, s>>>(m, X, N, u, derivs);
  return cudaGetLastError();
}

// Output block width: 16 RN >= the widest layer (RN a power of two, up to 16).
template <typename Tp, int RND, int NS>
static cudaError_t eval_launch(const MlpDev& m, const double* X, int64_t N, double* u, double* derivs,
                               cudaStream_t s) {
  if (m.d_in > kEvIn || m.max_w > 256) return cudaErrorInvalidValue;
  if (m.max_w <= 16) return eval_launch_rn<Tp, RND, NS, 1>(m, X, N, u, derivs, s);
  if (m.max_w <= 32) return eval_launch_rn<Tp, RND, NS, 2>(m, X, N, u, derivs, s);
  if (m.max_w <= 64) return eval_launch_rn<Tp, RND, NS, 4>(m, X, N, u, derivs, s);
  if (m.max_w <= 128) return eval_launch_rn<Tp, RND, NS, 8>(m, X, N, u, derivs, s);
  return eval_launch_rn<Tp, RND, NS, 16>(m, X, N, u, derivs, s);
}

cudaError_t launch_mlp_eval(const MlpDev& m, int prec, const double* X, int64_t N, double* u, double* derivs,
                            cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const bool d = derivs != nullptr;
  switch (prec) {
    case 0:
      return d ? eval_launch<double, 0, 4>(m, X, N, u, derivs, s) : eval_launch<double, 0, 1>(m, X, N, u, nullptr, s);
    case 1:
      return d ? eval_launch<float, 0, 4>(m, X, N, u, derivs, s) : eval_launch<float, 0, 1>(m, X, N, u, nullptr, s);
    case 2:
      if (tc_fits(m, true)) return launch_mlp_eval_tc(m, m.tc_packed, X, N, u, m.status, s, true);
      return eval_launch<float, 1, 1>(m, X, N, u, nullptr, s);
    case 3:
      if (tc_fits(m, false)) return launch_mlp_eval_tc(m, m.tc_packed, X, N, u, m.status, s, false);
      return eval_launch<float, 2, 1>(m, X, N, u, nullptr, s);
  }
  return cudaErrorInvalidValue;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

cudaError_t launch_f64_to_f32(const double* src, float* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  f64_to_f32_kernel<<<148, 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Training on CUDA cores: loss (Eqs. 11-14) and its gradient.
//   1. count points per loss term
//   2. forward (tiled GEMMs as in the evaluation, 16 points x 4 streams per
//      tile), storing (t, z_S, z_SS, z_tau) of every hidden layer and the
//      adjoint seeds dLoss/d(u, u_S, u_SS, u_tau)
//   3. adjoint (tiled GEMMs against W_l, top layer down), storing
//      dLoss/d(z, z_S, z_SS, z_tau) of every layer
//   4. weight gradient: for every layer a GEMM over points and streams of
//      dz_s (x) h_s, h_s rebuilt from the stored activations, split over
//      chunks of points whose partial sums are added into the gradient
// Workspace layout (Tp): act[l][p][s][o] for hidden layers, dz[l][p][s][o] for
// all layers (the seeds are dz of the output layer): a row (p, s) of a layer
// is its w_l neurons, contiguous.
// ---------------------------------------------------------------------------

static TrainLayout train_layout(const MlpDev& m, int64_t N) {
  TrainLayout L{};
  int64_t o = 0;
  for (int l = 1; l < m.n_lin; ++l) {
    L.act_off[l] = o;
    o += 4LL * m.widths[l] * N;
  }
  for (int l = 1; l <= m.n_lin; ++l) {
    L.dz_off[l] = o;
    o += 4LL * m.widths[l] * N;
  }
  L.total = o;
  return L;
}

// Workspace: activations and adjoints (the CUDA-core layout below, or the
// tensor-core path's own, whichever is larger), then the loss accumulators.
// The TF32 tensor-core path adds its packed W_l and W_l^T after the accumulators.
struct WsTail {
  size_t acc, pack, total;
};

static WsTail ws_tail(const MlpDev& m, const TrainLayout& L, size_t elem, int64_t N) {
  WsTail w;
  size_t body = (size_t)L.total * elem;
  const size_t tcb = train_tc_workspace_bytes(m, N);
  if (tcb > body) body = tcb;
  if (train_tf32_supported(m)) {  // FP32, the batch padded to 32-point tiles
    const size_t t32 = (size_t)train_layout(m, (N + 31) / 32 * 32).total * sizeof(float);
    if (t32 > body) body = t32;
  }
  w.acc = (body + 255) / 256 * 256;
  w.pack = w.acc + 256;
  w.total = w.pack + train_tf32_pack_bytes(m);
  return w;
}

size_t loss_grad_workspace_bytes(const MlpDev& m, int64_t N) {
  const TrainLayout L = train_layout(m, N);
  return ws_tail(m, L, sizeof(double), N).total + 256;  // + alignment of the caller's pointer
}

// Points per loss term; a kind outside 0..3, or 4 without values (data_ok
// false), is counted nowhere and recorded as BS_EINVAL in the status word.
__global__ void count_kinds_kernel(const int8_t* __restrict__ kind, int64_t N, unsigned long long* cnt, int data_ok,
                                   int* status) {
  unsigned long long c0 = 0, c1 = 0, c2 = 0;
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = kind[i];
    if (k == 0 || (k == 4 && data_ok)) ++c0;
    else if (k == 1 || k == 2) ++c1;
    else if (k == 3) ++c2;
    else bad = true;
  }
  for (int s = 16; s >= 1; s >>= 1) {
    c0 += __shfl_down_sync(kFull, c0, s);
    c1 += __shfl_down_sync(kFull, c1, s);
    c2 += __shfl_down_sync(kFull, c2, s);
  }
  bad = __any_sync(kFull, bad);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(cnt + 0, c0);
    atomicAdd(cnt + 1, c1);
    atomicAdd(cnt + 2, c2);
    if (bad && status != nullptr) atomicExch(status, 1);  // BS_EINVAL
  }
}

// Forward of a training step: the evaluation kernel's tiles (16 points x 4
// streams, rows (p, s) on adjacent rows), storing (t, z_S, z_SS, z_tau) of
// every hidden neuron, then the loss terms and adjoint seeds per point.
template <typename Tp, int RND, int RN>
__global__ void __launch_bounds__(kEvThreads) train_fwd_kernel(MlpDev m, LossArgs la, TrainLayout TL,
                                                               Tp* __restrict__ ws,
                                                               const unsigned long long* __restrict__ cnt,
                                                               double* __restrict__ loss_acc) {
  constexpr int WPAD = 16 * RN, WTS = WPAD + 4, PPT = kEvRows / 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double s_acc[3];
  Tp* H = reinterpret_cast<Tp*>(smraw);  // [WPAD][kEvRS] h of the tile, neuron-major
  Tp* Wt = H + hrows_size(WPAD);             // [kEvKC][WTS] staged weights
  Tp* Hin = Wt + kEvKC * WTS;            // [kEvIn][kEvRS] input streams
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
  const int r0 = rg * 4, c0 = cg * RN;
  const int64_t N = la.N;
  const int64_t p0 = (int64_t)blockIdx.x * PPT;
  if (tid < 3) s_acc[tid] = 0.0;
  for (int i = tid; i < kEvIn * kEvRows; i += kEvThreads) {
    const int k = i / kEvRows, r = i % kEvRows;
    const int st = r & 3;
    const int64_t p = p0 + (r >> 2);
    Tp v = (Tp)0;
    if (k < m.d_in && p < N) {
      const double sc = 2.0 / (m.hi[k] - m.lo[k]);
      if (st == 0) v = rop<RND>((Tp)(sc * (la.X[p * m.d_in + k] - m.lo[k]) - 1.0));
      else if (st == 1) v = k == 0 ? (Tp)sc : (Tp)0;
      else if (st == 3) v = k == 1 ? (Tp)sc : (Tp)0;
    }
    Hin[hrow(k) + r] = v;
  }
  const Tp* prm = params_of<Tp>(m);
  const int64_t pt = p0 + rg;  // this thread's point (its rows r0 .. r0 + 3 are the point's streams)
  for (int l = 1; l < m.n_lin; ++l) {
    const int wi = m.widths[l - 1], wo = m.widths[l];
    const Tp* Wl = prm + m.poff[l];
    const Tp* bl = Wl + (int64_t)wo * wi;
    const Tp* Hs = l == 1 ? Hin : H;
    Tp acc[4][RN];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < RN; ++q) acc[r][q] = (Tp)0;
    for (int kc = 0; kc < wi; kc += kEvKC) {
      const int kn = wi - kc < kEvKC ? wi - kc : kEvKC;
      __syncthreads();
      for (int i = tid; i < kEvKC * WPAD; i += kEvThreads) {
        const int o = i / kEvKC, k = i % kEvKC;
        Wt[k * WTS + o] = (k < kn && o < wo) ? rop<RND>(Wl[(int64_t)o * wi + kc + k]) : (Tp)0;
      }
      __syncthreads();
      for (int k = 0; k < kn; ++k) {
        Tp a[4], b[RN];
        load_vec<Tp, 4>(Hs + hrow(kc + k) + r0, a);
        load_vec<Tp, RN>(Wt + k * WTS + c0, b);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < RN; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
      }
    }
    __syncthreads();
    Tp* act = ws + TL.act_off[l];
#pragma unroll
    for (int q = 0; q < RN; ++q) {
      const int o = c0 + q;
      const bool ok = o < wo;
      const Tp z = acc[0][q] + (ok ? bl[o] : (Tp)0), zS = acc[1][q], zSS = acc[2][q], zT = acc[3][q];
      const Tp t = tanh_t<Tp>(z);
      const Tp d1 = (Tp)1 - t * t;
      store4<Tp>(H + hrow(o) + r0, ok ? rop<RND>(t) : (Tp)0, ok ? rop<RND>(d1 * zS) : (Tp)0,
                 ok ? rop<RND>(d1 * zSS - (Tp)2 * t * d1 * zS * zS) : (Tp)0, ok ? rop<RND>(d1 * zT) : (Tp)0);
      if (ok && pt < N) {
        act[(pt * 4 + 0) * wo + o] = t;
        act[(pt * 4 + 1) * wo + o] = zS;
        act[(pt * 4 + 2) * wo + o] = zSS;
        act[(pt * 4 + 3) * wo + o] = zT;
      }
    }
  }
  __syncthreads();
  // output layer (w -> 1, linear): four threads per row; the four rows of a
  // point end on lanes base, base + 4, base + 8, base + 12 of its 16 threads
  double sq[3] = {0.0, 0.0, 0.0};
  {
    const int wi = m.widths[m.n_lin - 1];
    const Tp* Wo = prm + m.poff[m.n_lin];
    const Tp* Hs = m.n_lin == 1 ? Hin : H;
    const int row = tid >> 2, part = tid & 3;
    Tp z = (Tp)0;
    for (int k = part; k < wi; k += 4) z = fma(rop<RND>(Wo[k]), Hs[hrow(k) + row], z);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    const int base = (tid & 31) & ~15;
    Tp out[4];
#pragma unroll
    for (int st = 0; st < 4; ++st) out[st] = __shfl_sync(0xffffffffu, z, base + 4 * st);
    out[0] += Wo[wi];
    const int64_t p = p0 + (tid >> 4);
    if ((tid & 15) == 0 && p < N) {
      const int kd = la.kind[p];
      double xin[8];
      for (int i = 0; i < m.d_in; ++i) xin[i] = la.X[p * m.d_in + i];
      double Ki, si, ri, tgt;
      point_setup(la, m.d_in, xin, kd, Ki, si, ri, tgt);
      const double S = xin[0];
      double gu = 0.0, gS = 0.0, gSS = 0.0, gT = 0.0;
      if (kd == 0) {
        const double f = (double)out[3] - 0.5 * si * si * S * S * (double)out[2] - ri * S * (double)out[1] +
                         ri * (double)out[0];
        sq[0] = f * f;
        const double gf = 2.0 * f / (double)cnt[0];
        gT = gf;
        gSS = -0.5 * si * si * S * S * gf;
        gS = -ri * S * gf;
        gu = ri * gf;
      } else if (kd == 4 && la.y != nullptr) {  // data point: misfit to its given value, in term 0
        const double e = (double)out[0] - la.y[p];
        sq[0] = e * e;
        gu = 2.0 * e / (double)cnt[0];
      } else if (kd >= 1 && kd <= 3) {
        const double e = (double)out[0] - tgt;
        const int tt = (kd == 3) ? 2 : 1;
        sq[tt] = e * e;
        gu = 2.0 * e / (double)cnt[tt];
      }
      Tp* dz = ws + TL.dz_off[m.n_lin];
      dz[p * 4 + 0] = (Tp)gu;
      dz[p * 4 + 1] = (Tp)gS;
      dz[p * 4 + 2] = (Tp)gSS;
      dz[p * 4 + 3] = (Tp)gT;
    }
  }
  if (sq[0] != 0.0) atomicAdd(&s_acc[0], sq[0]);
  if (sq[1] != 0.0) atomicAdd(&s_acc[1], sq[1]);
  if (sq[2] != 0.0) atomicAdd(&s_acc[2], sq[2]);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(loss_acc + 0, s_acc[0]);
    atomicAdd(loss_acc + 1, s_acc[1]);
    atomicAdd(loss_acc + 2, s_acc[2]);
  }
}

// Adjoint of a training step, top layer down, on the same tiles: the dz of
// layer l (neuron-major in shared memory, the GEMM's A) times W_l gives
// ah = W_l^T dz for the 4 streams of each point; the thread holding a point's
// rows combines them with that point's stored (t, z_S, z_SS, z_tau) into the
// dz of layer l - 1, written to the workspace and back over the tile.
template <typename Tp, int RND, int RN>
__global__ void __launch_bounds__(kEvThreads) train_bwd_kernel(MlpDev m, int64_t N, TrainLayout TL,
                                                               Tp* __restrict__ ws) {
  constexpr int WPAD = 16 * RN, WTS = WPAD + 4, PPT = kEvRows / 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  Tp* D = reinterpret_cast<Tp*>(smraw);  // [WPAD][kEvRS] dz of the current layer, neuron-major
  Tp* Wt = D + hrows_size(WPAD);             // [kEvKC][WTS] staged weights, W_l[kc + k][i] at [k][i]
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;
  const int r0 = rg * 4, c0 = cg * RN;
  const int64_t p0 = (int64_t)blockIdx.x * PPT;
  const int64_t pt = p0 + rg;
  const Tp* prm = params_of<Tp>(m);
  {  // the seeds: dz of the output layer (one neuron)
    const Tp* dzL = ws + TL.dz_off[m.n_lin];
    for (int r = tid; r < kEvRows; r += kEvThreads) {
      const int64_t p = p0 + (r >> 2);
      D[r] = p < N ? rop<RND>(dzL[p * 4 + (r & 3)]) : (Tp)0;
    }
  }
  for (int l = m.n_lin; l >= 2; --l) {
    const int wi = m.widths[l - 1], wo = m.widths[l];
    const Tp* Wl = prm + m.poff[l];
    Tp acc[4][RN];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < RN; ++q) acc[r][q] = (Tp)0;
    for (int kc = 0; kc < wo; kc += kEvKC) {
      const int kn = wo - kc < kEvKC ? wo - kc : kEvKC;
      __syncthreads();
      for (int i = tid; i < kEvKC * WPAD; i += kEvThreads) {
        const int k = i / WPAD, n = i % WPAD;
        Wt[k * WTS + n] = (k < kn && n < wi) ? rop<RND>(Wl[(int64_t)(kc + k) * wi + n]) : (Tp)0;
      }
      __syncthreads();
      for (int k = 0; k < kn; ++k) {
        Tp a[4], b[RN];
        load_vec<Tp, 4>(D + hrow(kc + k) + r0, a);
        load_vec<Tp, RN>(Wt + k * WTS + c0, b);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < RN; ++q) acc[r][q] = fma(a[r], b[q], acc[r][q]);
      }
    }
    __syncthreads();  // every thread has read this layer's dz before it is overwritten
    const Tp* act = ws + TL.act_off[l - 1];
    Tp* dzp = ws + TL.dz_off[l - 1];
#pragma unroll
    for (int q = 0; q < RN; ++q) {
      const int i = c0 + q;
      const bool ok = i < wi && pt < N;
      const Tp ah = acc[0][q], ahS = acc[1][q], ahSS = acc[2][q], ahT = acc[3][q];
      const Tp t = ok ? act[(pt * 4 + 0) * wi + i] : (Tp)0;
      const Tp zs = ok ? act[(pt * 4 + 1) * wi + i] : (Tp)0;
      const Tp zss = ok ? act[(pt * 4 + 2) * wi + i] : (Tp)0;
      const Tp zt = ok ? act[(pt * 4 + 3) * wi + i] : (Tp)0;
      const Tp d1 = (Tp)1 - t * t, d2 = (Tp)-2 * t * d1;
      Tp bar_d1 = ahS * zs + ahSS * zss + ahT * zt;
      const Tp bar_d2 = ahSS * zs * zs;
      Tp bar_t = ah;
      bar_t += (Tp)-2 * d1 * bar_d2;
      bar_d1 += (Tp)-2 * t * bar_d2;
      bar_t += (Tp)-2 * t * bar_d1;
      Tp g[4];
      g[0] = d1 * bar_t;
      g[1] = ahS * d1 + (Tp)2 * ahSS * d2 * zs;
      g[2] = ahSS * d1;
      g[3] = ahT * d1;
      if (!ok) g[0] = g[1] = g[2] = g[3] = (Tp)0;
      if (ok) {
#pragma unroll
        for (int st = 0; st < 4; ++st) dzp[(pt * 4 + st) * wi + i] = g[st];
      }
      store4<Tp>(D + hrow(i) + r0, rop<RND>(g[0]), rop<RND>(g[1]), rop<RND>(g[2]), rop<RND>(g[3]));
    }
  }
}

// Weight gradient of layer l as a GEMM over rows (points x streams):
// gW[o][i] = sum over rows of dz_l[row][o] h_{l-1}[row][i], h rebuilt from the
// stored (t, z_S, z_SS, z_tau) (layer 1: from the inputs).  A CTA of 256
// threads owns a 64 x 64 block of (o, i) for one chunk of kWgRows rows, staged
// 32 rows at a time; thread (ty, tx) accumulates o = 4 ty .. + 3 against
// i = 4 tx .. + 3 and adds its partial sums into the FP64 gradient.
constexpr int kWgRows = 2048;
constexpr int kWgStride = 64 + 4;

template <typename Tp, int RND>
__global__ void __launch_bounds__(256) train_wgrad_kernel(MlpDev m, LossArgs la, TrainLayout TL,
                                                          const Tp* __restrict__ ws, int l,
                                                          double* __restrict__ grad) {
  __shared__ __align__(16) Tp sDZ[32][kWgStride];
  __shared__ __align__(16) Tp sH[32][kWgStride];
  const int wi = m.widths[l - 1], wo = m.widths[l];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int ob = blockIdx.y * 64, ib = blockIdx.x * 64;
  const int64_t rows = 4 * la.N;
  const int64_t rb = (int64_t)blockIdx.z * kWgRows;
  const int64_t re = rb + kWgRows < rows ? rb + kWgRows : rows;
  const Tp* dz = ws + TL.dz_off[l];
  const Tp* act = l >= 2 ? ws + TL.act_off[l - 1] : nullptr;
  Tp acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (Tp)0;
  for (int64_t r32 = rb; r32 < re; r32 += 32) {
    __syncthreads();
    for (int q = tid; q < 32 * 64; q += 256) {  // dz rows, coalesced along o
      const int k = q / 64, o = q % 64;
      const int64_t row = r32 + k;
      sDZ[k][o] = (row < re && ob + o < wo) ? rop<RND>(dz[row * wo + ob + o]) : (Tp)0;
    }
    for (int q = tid; q < 8 * 64; q += 256) {  // h of 8 points x 64 inputs, 4 streams each
      const int pp = q / 64, i = q % 64, ig = ib + i;
      const int64_t p = (r32 >> 2) + pp;
      Tp h0 = 0, h1 = 0, h2 = 0, h3 = 0;
      if (4 * p < re && ig < wi) {
        if (l >= 2) {
          const Tp t = act[(p * 4 + 0) * wi + ig], zs = act[(p * 4 + 1) * wi + ig];
          const Tp zss = act[(p * 4 + 2) * wi + ig], zt = act[(p * 4 + 3) * wi + ig];
          const Tp d1 = (Tp)1 - t * t;
          h0 = t;
          h1 = d1 * zs;
          h2 = d1 * zss - (Tp)2 * t * d1 * zs * zs;
          h3 = d1 * zt;
        } else {
          const double sc = 2.0 / (m.hi[ig] - m.lo[ig]);
          h0 = (Tp)(sc * (la.X[p * m.d_in + ig] - m.lo[ig]) - 1.0);
          h1 = (Tp)(ig == 0 ? sc : 0.0);
          h3 = (Tp)(ig == 1 ? sc : 0.0);
        }
      }
      sH[pp * 4 + 0][i] = rop<RND>(h0);
      sH[pp * 4 + 1][i] = rop<RND>(h1);
      sH[pp * 4 + 2][i] = rop<RND>(h2);
      sH[pp * 4 + 3][i] = rop<RND>(h3);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      Tp a[4], b[4];
      load_vec<Tp, 4>(&sDZ[k][ty * 4], a);
      load_vec<Tp, 4>(&sH[k][tx * 4], b);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
  }
  double* g = grad + m.poff[l];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int o = ob + ty * 4 + x;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = ib + tx * 4 + y;
      if (o < wo && i < wi) atomicAdd(g + (int64_t)o * wi + i, (double)acc[x][y]);
    }
  }
}

// Bias gradient of layer l: gb[o] = sum over points of dz_l[(p, 0)][o] (the
// value stream), one thread per o over a chunk of points.
template <typename Tp, int RND>
__global__ void train_bgrad_kernel(MlpDev m, int64_t N, TrainLayout TL, const Tp* __restrict__ ws, int l,
                                   double* __restrict__ grad, int64_t chunk) {
  const int wi = m.widths[l - 1], wo = m.widths[l];
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= wo) return;
  const int64_t pb = (int64_t)blockIdx.y * chunk;
  const int64_t pe = pb + chunk < N ? pb + chunk : N;
  const Tp* dz = ws + TL.dz_off[l];
  Tp acc = (Tp)0;
  for (int64_t p = pb; p < pe; ++p) acc += rop<RND>(dz[(p * 4) * wo + o]);
  atomicAdd(grad + m.poff[l] + (int64_t)wo * wi + o, (double)acc);
}

__global__ void loss_finish_kernel(const double* acc, const unsigned long long* cnt, double* loss3) {
  if (threadIdx.x == 0) {
    loss3[0] = cnt[0] ? acc[0] / (double)cnt[0] : 0.0;
    loss3[1] = cnt[1] ? acc[1] / (double)cnt[1] : 0.0;
    loss3[2] = cnt[2] ? acc[2] / (double)cnt[2] : 0.0;
  }
}

template <typename Tp, int RND, int RN>
static cudaError_t simt_train_launch(const MlpDev& m, const LossArgs& la, const TrainLayout& TL, Tp* ws,
                                     const unsigned long long* cnt, double* acc, double* grad, cudaStream_t s) {
  const size_t smem = eval_smem_bytes<Tp>(RN);
  cudaError_t e = cudaFuncSetAttribute(train_fwd_kernel<Tp, RND, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(train_bwd_kernel<Tp, RND, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned tiles = (unsigned)((la.N + kEvRows / 4 - 1) / (kEvRows / 4));
  train_fwd_kernel<Tp, RND, RN><<<tiles, kEvThreads, smem, s>>>(m, la, TL, ws, cnt, acc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  train_bwd_kernel<Tp, RND, RN><<<tiles, kEvThreads, smem, s>>>(m, la.N, TL, ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned nz = (unsigned)((4 * la.N + kWgRows - 1) / kWgRows);
  const int64_t bchunk = 1024;
  for (int l = 1; l <= m.n_lin; ++l) {
    const int wi = m.widths[l - 1], wo = m.widths[l];
    train_wgrad_kernel<Tp, RND><<<dim3((wi + 63) / 64, (wo + 63) / 64, nz), 256, 0, s>>>(m, la, TL, ws, l, grad);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    train_bgrad_kernel<Tp, RND><<<dim3((wo + 127) / 128, (unsigned)((la.N + bchunk - 1) / bchunk)), 128, 0, s>>>(
        m, la.N, TL, ws, l, grad, bchunk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename Tp, int RND>
static cudaError_t loss_grad_impl(const MlpDev& m, const LossArgs& la, double* loss3, double* grad, void* workspace,
                                  size_t ws_bytes, cudaStream_t s) {
  const TrainLayout TL = train_layout(m, la.N);
  const WsTail WT = ws_tail(m, TL, sizeof(Tp), la.N);
  if (WT.total > ws_bytes) return cudaErrorInvalidValue;
  Tp* ws = reinterpret_cast<Tp*>(workspace);
  unsigned char* base = reinterpret_cast<unsigned char*>(workspace);
  // small accumulators live after the activations
  unsigned char* tail = base + WT.acc;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(tail);
  double* acc = reinterpret_cast<double*>(tail + 24);
  cudaError_t e = cudaMemsetAsync(tail, 0, 48, s);
  if (e != cudaSuccess) return e;
  if (RND == 2 && train_tc_supported(m)) {  // BF16 on the tensor cores (zeroes grad, counts, finishes loss3)
    if (((uintptr_t)base & 255) != 0) return cudaErrorInvalidValue;
    return launch_train_tc(m, la, base, cnt, acc, grad, loss3, s);
  }
  int64_t np = 0;
  for (int l = 1; l <= m.n_lin; ++l) np += (int64_t)m.widths[l] * m.widths[l - 1] + m.widths[l];
  e = cudaMemsetAsync(grad, 0, (size_t)np * sizeof(double), s);
  if (e != cudaSuccess) return e;
  count_kinds_kernel<<<148, 256, 0, s>>>(la.kind, la.N, cnt, la.y != nullptr, m.status);
  if (RND == 1 && sizeof(Tp) == 4 && train_tf32_supported(m)) {  // TF32 on the tensor cores
    const TrainLayout TLp = train_layout(m, (la.N + 31) / 32 * 32);
    e = launch_train_tf32(m, la, reinterpret_cast<float*>(workspace), TLp, base + WT.pack, cnt, acc, grad, s);
    if (e != cudaSuccess) return e;
    loss_finish_kernel<<<1, 32, 0, s>>>(acc, cnt, loss3);
    return cudaGetLastError();
  }
  // CUDA cores: forward, adjoint, per-layer weight and bias gradients
  if (m.max_w <= 16) e = simt_train_launch<Tp, RND, 1>(m, la, TL, ws, cnt, acc, grad, s);
  else if (m.max_w <= 32) e = simt_train_launch<Tp, RND, 2>(m, la, TL, ws, cnt, acc, grad, s);
  else if (m.max_w <= 64) e = simt_train_launch<Tp, RND, 4>(m, la, TL, ws, cnt, acc, grad, s);
  else if (m.max_w <= 128) e = simt_train_launch<Tp, RND, 8>(m, la, TL, ws, cnt, acc, grad, s);
  else e = simt_train_launch<Tp, RND, 16>(m, la, TL, ws, cnt, acc, grad, s);
  if (e != cudaSuccess) return e;
  loss_finish_kernel<<<1, 32, 0, s>>>(acc, cnt, loss3);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(const MlpDev& m, const LossArgs& la, double* loss3, double* grad, void* workspace,
                             size_t ws_bytes, cudaStream_t s) {
  switch (la.prec) {
    case 0:
      return loss_grad_impl<double, 0>(m, la, loss3, grad, workspace, ws_bytes, s);
    case 1:
      return loss_grad_impl<float, 0>(m, la, loss3, grad, workspace, ws_bytes, s);
    case 2:
      return loss_grad_impl<float, 1>(m, la, loss3, grad, workspace, ws_bytes, s);
    case 3:
      return loss_grad_impl<float, 2>(m, la, loss3, grad, workspace, ws_bytes, s);
  }
  return cudaErrorInvalidValue;
}

// Adam (Kingma & Ba) on the FP64 master parameters; refreshes the FP32 copy.
// ic1, ic2: reciprocals of the bias corrections 1 - b1^t, 1 - b2^t (formed once
// on the host: FP64 division is a long instruction sequence on this part).
__global__ void adam_kernel(int64_t n, double* __restrict__ th, double* __restrict__ m1, double* __restrict__ m2,
                            const double* __restrict__ g, double ic1, double ic2, double lr, float* __restrict__ p32) {
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double gi = g[i];
    const double a = b1 * m1[i] + (1.0 - b1) * gi;
    const double v = b2 * m2[i] + (1.0 - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const double mh = a * ic1, vh = v * ic2;
    const double t = th[i] - lr * mh / (sqrt(vh) + eps);
    th[i] = t;
    p32[i] = (float)t;
  }
}

cudaError_t launch_adam(int64_t n, double* theta, double* mom1, double* mom2, const double* g, int step, double lr,
                        float* p32, cudaStream_t s) {
  const double c1 = 1.0 - pow(0.9, (double)step), c2 = 1.0 - pow(0.999, (double)step);
  adam_kernel<<<148, 256, 0, s>>>(n, theta, mom1, mom2, g, 1.0 / c1, 1.0 / c2, lr, p32);
  return cudaGetLastError();
}

}  // namespace bsp
