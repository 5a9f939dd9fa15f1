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
// Evaluation: one thread per point, activation columns in shared memory.
// ---------------------------------------------------------------------------
template <typename Tp, int RND, int NS>
__global__ void mlp_eval_kernel(MlpDev m, const double* __restrict__ X, int64_t N, double* __restrict__ u,
                                double* __restrict__ derivs) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Tp* sh = reinterpret_cast<Tp*>(smraw);
  const int TP = blockDim.x, tid = threadIdx.x, W = m.max_w;
  const int64_t p = (int64_t)blockIdx.x * TP + tid;
  const bool valid = p < N;
  // buffers [buf][stream][i][tid]
  auto col = [&](int buf, int s, int i) -> Tp& { return sh[(((int64_t)buf * NS + s) * W + i) * TP + tid]; };
  double xin[8];
  for (int i = 0; i < m.d_in; ++i) xin[i] = valid ? X[p * m.d_in + i] : 0.0;
  if (NS == 4)
    input_streams<Tp>(m, xin, &col(0, 0, 0), &col(0, 1, 0), &col(0, 2, 0), &col(0, 3, 0), TP);
  else
    input_streams<Tp>(m, xin, &col(0, 0, 0), (Tp*)nullptr, (Tp*)nullptr, (Tp*)nullptr, TP);
  if (RND != 0)
    for (int i = 0; i < m.d_in; ++i) col(0, 0, i) = rop<RND>(col(0, 0, i));
  const Tp* prm = params_of<Tp>(m);
  int cur = 0;
  for (int l = 1; l <= m.n_lin; ++l) {
    const int wi = m.widths[l - 1], wo = m.widths[l];
    const Tp* Wl = prm + m.poff[l];
    const Tp* bl = Wl + (int64_t)wo * wi;
    const bool last = l == m.n_lin;
    for (int o = 0; o < wo; ++o) {
      Tp z = 0, zS = 0, zSS = 0, zT = 0;
      const Tp* wr = Wl + (int64_t)o * wi;
      for (int i = 0; i < wi; ++i) {
        const Tp w = rop<RND>(__ldg(wr + i));
        z = fma(w, col(cur, 0, i), z);
        if (NS == 4) {
          zS = fma(w, col(cur, 1, i), zS);
          zSS = fma(w, col(cur, 2, i), zSS);
          zT = fma(w, col(cur, 3, i), zT);
        }
      }
      z += __ldg(bl + o);
      if (!last) {
        const Tp t = tanh_t<Tp>(z);
        col(cur ^ 1, 0, o) = rop<RND>(t);
        if (NS == 4) {
          const Tp d1 = (Tp)1 - t * t;
          col(cur ^ 1, 1, o) = rop<RND>(d1 * zS);
          col(cur ^ 1, 2, o) = rop<RND>(d1 * zSS - (Tp)2 * t * d1 * zS * zS);
          col(cur ^ 1, 3, o) = rop<RND>(d1 * zT);
        }
      } else if (valid) {
        u[p] = (double)z;
        if (NS == 4 && derivs) {
          derivs[3 * p + 0] = (double)zS;
          derivs[3 * p + 1] = (double)zSS;
          derivs[3 * p + 2] = (double)zT;
        }
      }
    }
    cur ^= 1;
  }
}

static int points_per_cta(size_t per_thread) {
  int TP = (int)((160 * 1024) / per_thread);
  if (TP >= 128) return 128;
  if (TP >= 32) return (TP / 32) * 32;
  int q = 1;
  while (q * 2 <= TP) q *= 2;
  return q;
}

template <typename Tp, int RND, int NS>
static cudaError_t eval_launch(const MlpDev& m, const double* X, int64_t N, double* u, double* derivs,
                               cudaStream_t s) {
  const size_t per_thread = 2 * (size_t)NS * m.max_w * sizeof(Tp);
  const int TP = points_per_cta(per_thread);
  const size_t smem = per_thread * TP;
  cudaError_t e = cudaFuncSetAttribute(mlp_eval_kernel<Tp, RND, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (N + TP - 1) / TP;
  mlp_eval_kernel<Tp, RND, NS><<<(unsigned)blocks, TP, smem, s>>>(m, X, N, u, derivs);
  return cudaGetLastError();
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
// Training: loss (Eqs. 11-14) and its gradient.
//   1. count points per loss term
//   2. forward per point, storing (t, z_S, z_SS, z_tau) of every hidden layer
//      and the adjoint seeds dLoss/d(u, u_S, u_SS, u_tau)
//   3. adjoint per point, storing dLoss/d(z, z_S, z_SS, z_tau) of every layer
//   4. weight gradient: for every layer a reduction over points and streams of
//      dz_s (x) h_s, with h_s rebuilt from the stored activations
// Workspace layout (Tp): act[l][s][o][p] for hidden layers, dz[l][s][o][p] for
// all layers (the seeds are dz of the output layer).
// ---------------------------------------------------------------------------

struct TrainLayout {
  int64_t act_off[16];  // offsets (elements) of act[l], l = 1..n_lin-1
  int64_t dz_off[16];   // offsets of dz[l], l = 1..n_lin
  int64_t total;        // elements
};

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
struct WsTail {
  size_t acc, total;
};

static WsTail ws_tail(const MlpDev& m, const TrainLayout& L, size_t elem, int64_t N) {
  WsTail w;
  size_t body = (size_t)L.total * elem;
  const size_t tcb = train_tc_workspace_bytes(m, N);
  if (tcb > body) body = tcb;
  w.acc = (body + 255) / 256 * 256;
  w.total = w.acc + 64;
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

template <typename Tp, int RND>
__global__ void train_fwd_kernel(MlpDev m, LossArgs la, TrainLayout TL, Tp* __restrict__ ws,
                                 const unsigned long long* __restrict__ cnt, double* __restrict__ loss_acc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double s_acc[3];
  Tp* sh = reinterpret_cast<Tp*>(smraw);
  const int TP = blockDim.x, tid = threadIdx.x, W = m.max_w;
  const int64_t N = la.N;
  const int64_t p = (int64_t)blockIdx.x * TP + tid;
  const bool valid = p < N;
  auto col = [&](int buf, int s, int i) -> Tp& { return sh[(((int64_t)buf * 4 + s) * W + i) * TP + tid]; };
  double xin[8];
  for (int i = 0; i < m.d_in; ++i) xin[i] = valid ? la.X[p * m.d_in + i] : 0.0;
  input_streams<Tp>(m, xin, &col(0, 0, 0), &col(0, 1, 0), &col(0, 2, 0), &col(0, 3, 0), TP);
  if (RND != 0)
    for (int i = 0; i < m.d_in; ++i) col(0, 0, i) = rop<RND>(col(0, 0, i));
  const Tp* prm = params_of<Tp>(m);
  int cur = 0;
  Tp out[4] = {0, 0, 0, 0};
  for (int l = 1; l <= m.n_lin; ++l) {
    const int wi = m.widths[l - 1], wo = m.widths[l];
    const Tp* Wl = prm + m.poff[l];
    const Tp* bl = Wl + (int64_t)wo * wi;
    const bool last = l == m.n_lin;
    for (int o = 0; o < wo; ++o) {
      Tp z = 0, zS = 0, zSS = 0, zT = 0;
      const Tp* wr = Wl + (int64_t)o * wi;
      for (int i = 0; i < wi; ++i) {
        const Tp w = rop<RND>(__ldg(wr + i));
        z = fma(w, col(cur, 0, i), z);
        zS = fma(w, col(cur, 1, i), zS);
        zSS = fma(w, col(cur, 2, i), zSS);
        zT = fma(w, col(cur, 3, i), zT);
      }
      z += __ldg(bl + o);
      if (!last) {
        const Tp t = tanh_t<Tp>(z);
        const Tp d1 = (Tp)1 - t * t;
        col(cur ^ 1, 0, o) = rop<RND>(t);
        col(cur ^ 1, 1, o) = rop<RND>(d1 * zS);
        col(cur ^ 1, 2, o) = rop<RND>(d1 * zSS - (Tp)2 * t * d1 * zS * zS);
        col(cur ^ 1, 3, o) = rop<RND>(d1 * zT);
        if (valid) {
          Tp* a = ws + TL.act_off[l];
          a[(0 * (int64_t)wo + o) * N + p] = t;
          a[(1 * (int64_t)wo + o) * N + p] = zS;
          a[(2 * (int64_t)wo + o) * N + p] = zSS;
          a[(3 * (int64_t)wo + o) * N + p] = zT;
        }
      } else {
        out[0] = z;
        out[1] = zS;
        out[2] = zSS;
        out[3] = zT;
      }
    }
    cur ^= 1;
  }
  // loss terms and seeds
  double sq[3] = {0.0, 0.0, 0.0};
  if (valid) {
    const int kd = la.kind[p];
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
    dz[0 * N + p] = (Tp)gu;
    dz[1 * N + p] = (Tp)gS;
    dz[2 * N + p] = (Tp)gSS;
    dz[3 * N + p] = (Tp)gT;
  }
  // block sum through shared atomics (the CTA may be narrower than a warp)
  if (tid == 0) s_acc[0] = s_acc[1] = s_acc[2] = 0.0;
  __syncthreads();
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

// Adjoint per point: dz of layer l -> dz of layer l-1 through W_l^T and tanh.
template <typename Tp, int RND>
__global__ void train_bwd_kernel(MlpDev m, int64_t N, TrainLayout TL, Tp* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Tp* sh = reinterpret_cast<Tp*>(smraw);
  const int TP = blockDim.x, tid = threadIdx.x, W = m.max_w;
  const int64_t p = (int64_t)blockIdx.x * TP + tid;
  const bool valid = p < N;
  auto col = [&](int s, int i) -> Tp& { return sh[((int64_t)s * W + i) * TP + tid]; };
  const Tp* prm = params_of<Tp>(m);
  for (int l = m.n_lin; l >= 2; --l) {
    const int wi = m.widths[l - 1], wo = m.widths[l];
    const Tp* dzl = ws + TL.dz_off[l];
    for (int o = 0; o < wo; ++o)
      for (int s = 0; s < 4; ++s) col(s, o) = valid ? rop<RND>(dzl[((int64_t)s * wo + o) * N + p]) : (Tp)0;
    const Tp* Wl = prm + m.poff[l];
    const Tp* act = ws + TL.act_off[l - 1];
    Tp* dzp = ws + TL.dz_off[l - 1];
    for (int i = 0; i < wi; ++i) {
      Tp ah = 0, ahS = 0, ahSS = 0, ahT = 0;
      for (int o = 0; o < wo; ++o) {
        const Tp w = rop<RND>(__ldg(Wl + (int64_t)o * wi + i));
        ah = fma(w, col(0, o), ah);
        ahS = fma(w, col(1, o), ahS);
        ahSS = fma(w, col(2, o), ahSS);
        ahT = fma(w, col(3, o), ahT);
      }
      if (!valid) continue;
      const Tp t = act[(0 * (int64_t)wi + i) * N + p];
      const Tp zs = act[(1 * (int64_t)wi + i) * N + p];
      const Tp zss = act[(2 * (int64_t)wi + i) * N + p];
      const Tp zt = act[(3 * (int64_t)wi + i) * N + p];
      const Tp d1 = (Tp)1 - t * t, d2 = (Tp)-2 * t * d1;
      Tp bar_d1 = ahS * zs + ahSS * zss + ahT * zt;
      const Tp bar_d2 = ahSS * zs * zs;
      Tp bar_t = ah;
      bar_t += (Tp)-2 * d1 * bar_d2;
      bar_d1 += (Tp)-2 * t * bar_d2;
      bar_t += (Tp)-2 * t * bar_d1;
      dzp[(0 * (int64_t)wi + i) * N + p] = d1 * bar_t;
      dzp[(1 * (int64_t)wi + i) * N + p] = ahS * d1 + (Tp)2 * ahSS * d2 * zs;
      dzp[(2 * (int64_t)wi + i) * N + p] = ahSS * d1;
      dzp[(3 * (int64_t)wi + i) * N + p] = ahT * d1;
    }
    __syncthreads();
  }
}

// Weight gradient of layer l: gW[o][i] = sum_p sum_s dz_s[o][p] h_s[i][p],
// gb[o] = sum_p dz_0[o][p].  One CTA per (o-tile, i-tile, point chunk);
// 16x16 outputs per CTA, one per thread, FP64 atomics into the gradient.
template <typename Tp, int RND>
__global__ void grad_reduce_kernel(MlpDev m, LossArgs la, TrainLayout TL, const Tp* __restrict__ ws, int l,
                                   double* __restrict__ grad, int64_t chunk) {
  const int wi = m.widths[l - 1], wo = m.widths[l];
  const int64_t N = la.N;
  const int o = blockIdx.y * 16 + threadIdx.y;
  const int i = blockIdx.x * 16 + threadIdx.x;  // i == wi is the bias column
  const int64_t p0 = (int64_t)blockIdx.z * chunk;
  const int64_t p1 = min(N, p0 + chunk);
  __shared__ Tp sdz[4][16][33];
  __shared__ Tp shh[4][16][33];
  Tp acc = 0;
  const Tp* dz = ws + TL.dz_off[l];
  const Tp* act = (l >= 2) ? ws + TL.act_off[l - 1] : nullptr;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int64_t pb = p0; pb < p1; pb += 32) {
    // stage dz for 16 outputs x 32 points and h streams for 16 inputs x 32 points
    for (int q = ty * 16 + tx; q < 16 * 32; q += 256) {
      const int oo = q / 32, pp = q % 32;
      const int64_t pg = pb + pp;
      const int og = blockIdx.y * 16 + oo;
      for (int s = 0; s < 4; ++s)
        sdz[s][oo][pp] = (pg < p1 && og < wo) ? rop<RND>(dz[((int64_t)s * wo + og) * N + pg]) : (Tp)0;
      const int ig = blockIdx.x * 16 + oo;
      Tp h0 = 0, h1 = 0, h2 = 0, h3 = 0;
      if (pg < p1) {
        if (ig == wi) {
          h0 = 1;  // bias column: only the value stream
        } else if (ig < wi) {
          if (l >= 2) {
            const Tp t = act[((int64_t)0 * wi + ig) * N + pg];
            const Tp zs = act[((int64_t)1 * wi + ig) * N + pg];
            const Tp zss = act[((int64_t)2 * wi + ig) * N + pg];
            const Tp zt = act[((int64_t)3 * wi + ig) * N + pg];
            const Tp d1 = (Tp)1 - t * t;
            h0 = t;
            h1 = d1 * zs;
            h2 = d1 * zss - (Tp)2 * t * d1 * zs * zs;
            h3 = d1 * zt;
          } else {
            const double sc = 2.0 / (m.hi[ig] - m.lo[ig]);
            h0 = (Tp)(sc * (la.X[pg * m.d_in + ig] - m.lo[ig]) - 1.0);
            h1 = (Tp)((ig == 0) ? sc : 0.0);
            h2 = 0;
            h3 = (Tp)((ig == 1) ? sc : 0.0);
          }
        }
      }
      shh[0][oo][pp] = rop<RND>(h0);
      shh[1][oo][pp] = rop<RND>(h1);
      shh[2][oo][pp] = rop<RND>(h2);
      shh[3][oo][pp] = rop<RND>(h3);
    }
    __syncthreads();
#pragma unroll 4
    for (int pp = 0; pp < 32; ++pp) {
      acc = fma(sdz[0][ty][pp], shh[0][tx][pp], acc);
      acc = fma(sdz[1][ty][pp], shh[1][tx][pp], acc);
      acc = fma(sdz[2][ty][pp], shh[2][tx][pp], acc);
      acc = fma(sdz[3][ty][pp], shh[3][tx][pp], acc);
    }
    __syncthreads();
  }
  if (o < wo && i <= wi) {
    double* g = grad + m.poff[l];
    if (i < wi) atomicAdd(g + (int64_t)o * wi + i, (double)acc);
    else atomicAdd(g + (int64_t)wo * wi + o, (double)acc);
  }
}

__global__ void loss_finish_kernel(const double* acc, const unsigned long long* cnt, double* loss3) {
  if (threadIdx.x == 0) {
    loss3[0] = cnt[0] ? acc[0] / (double)cnt[0] : 0.0;
    loss3[1] = cnt[1] ? acc[1] / (double)cnt[1] : 0.0;
    loss3[2] = cnt[2] ? acc[2] / (double)cnt[2] : 0.0;
  }
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
  {  // CUDA cores: forward, adjoint, per-layer reductions
    {
      const size_t per_thread = 2 * 4 * (size_t)m.max_w * sizeof(Tp);
      const int TP = points_per_cta(per_thread);
      const size_t smem = per_thread * TP;
      e = cudaFuncSetAttribute(train_fwd_kernel<Tp, RND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      train_fwd_kernel<Tp, RND><<<(unsigned)((la.N + TP - 1) / TP), TP, smem, s>>>(m, la, TL, ws, cnt, acc);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    {
      const size_t per_thread = 4 * (size_t)m.max_w * sizeof(Tp);
      const int TP = points_per_cta(per_thread);
      const size_t smem = per_thread * TP;
      e = cudaFuncSetAttribute(train_bwd_kernel<Tp, RND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      train_bwd_kernel<Tp, RND><<<(unsigned)((la.N + TP - 1) / TP), TP, smem, s>>>(m, la.N, TL, ws);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t chunk = 2048;
    const unsigned nz = (unsigned)((la.N + chunk - 1) / chunk);
    for (int l = 1; l <= m.n_lin; ++l) {
      const int wi = m.widths[l - 1], wo = m.widths[l];
      dim3 grid((wi + 1 + 15) / 16, (wo + 15) / 16, nz);
      grad_reduce_kernel<Tp, RND><<<grid, dim3(16, 16), 0, s>>>(m, la, TL, ws, l, grad, chunk);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
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
