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
  int nb;       // 64-point blocks
  int per_cta;  // chunks per CTA along K
  float* partial;  // [gridDim.y][w][w]
  int* status;
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 q = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&q);
}

__global__ void __launch_bounds__(128) wgrad_tc_kernel(WgArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int w = a.w, t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int ot = blockIdx.x;
  constexpr uint32_t a_bytes = 128 * kChunk * 2;
  const uint32_t b_bytes = (uint32_t)w * kChunk * 2;
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
  while ((int)ncols < w) ncols <<= 1;
  if (warp == 0) tmem_alloc(tslot, ncols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc_bf16(w);
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
        const float* src = a.dz + ((int64_t)s * w + o) * N + pb;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = pb + e < N ? __ldg(src + e) : 0.0f;
        q = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
      }
      *reinterpret_cast<uint4*>(stA(st) + canon_off(row, kc * 8, kChunk)) = q;
    }
    // B: w rows (i) x 64 points of h_s rebuilt from the stored streams, BF16
    for (int it = t; it < w * (kChunk / 8); it += 128) {
      const int i = it >> 3, kc = it & 7;
      const int64_t pb = p0 + kc * 8;
      const float* t0 = a.act + ((int64_t)0 * w + i) * N + pb;
      const float* zs = a.act + ((int64_t)1 * w + i) * N + pb;
      const float* zx = a.act + ((int64_t)(s == 3 ? 3 : 2) * w + i) * N + pb;
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float h = 0.0f;
        if (pb + e < N) {
          const float tt = __ldg(t0 + e);
          const float d1 = 1.0f - tt * tt;
          if (s == 0) {
            h = tt;
          } else if (s == 1) {
            h = d1 * __ldg(zs + e);
          } else if (s == 2) {
            const float z1 = __ldg(zs + e);
            h = d1 * __ldg(zx + e) - 2.0f * tt * d1 * z1 * z1;
          } else {
            h = d1 * __ldg(zx + e);
          }
        }
        v[e] = h;
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
    float* dst = a.partial + ((int64_t)blockIdx.y * w + o) * w;
    for (int cc = 0; cc < w; cc += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
      if (o < w) {
#pragma unroll
        for (int e = 0; e < 32; e += 4)
          *reinterpret_cast<float4*>(dst + cc + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (s_fail && t == 0) atomicExch(a.status, 6);  // BS_TIMEOUT
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// gW[o][i] = sum over CTAs of the partial sums (FP64 accumulation).
__global__ void wgrad_sum_kernel(const float* __restrict__ partial, int ny, int w, double* __restrict__ gW) {
  const int64_t ww = (int64_t)w * w;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ww; q += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int y = 0; y < ny; ++y) acc += (double)partial[(int64_t)y * ww + q];
    gW[q] = acc;
  }
}

// gb[o] = sum_p dz_0[o][p], the adjoint rounded to BF16 like the GEMM operand.
__global__ void bias_grad_kernel(const float* __restrict__ dz, int64_t N, double* __restrict__ gb) {
  __shared__ double red[4];
  const int o = blockIdx.x, t = threadIdx.x;
  double acc = 0.0;
  for (int64_t p = t; p < N; p += blockDim.x)
    acc += (double)__bfloat162float(__float2bfloat16_rn(dz[(int64_t)o * N + p]));
  for (int s = 16; s >= 1; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
  if ((t & 31) == 0) red[t >> 5] = acc;
  __syncthreads();
  if (t == 0) gb[o] = red[0] + red[1] + red[2] + red[3];
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

size_t wgrad_smem_bytes(int w) { return 2 * (size_t)128 * kChunk * 2 + 2 * (size_t)w * kChunk * 2 + 64; }

}  // namespace

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
  return (size_t)ny * m.widths[1] * m.widths[1] * sizeof(float);
}

cudaError_t launch_wgrad_tc(const MlpDev& m, int64_t N, const float* dz, const float* act, double* gW, double* gb,
                            float* partial, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int w = m.widths[1];
  int ot, pc, ny;
  wgrad_grid(w, N, &ot, &pc, &ny);
  WgArgs a{dz, act, N, w, (int)((N + kChunk - 1) / kChunk), pc, partial, m.status};
  const size_t smem = wgrad_smem_bytes(w);
  cudaError_t e = cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  wgrad_tc_kernel<<<dim3(ot, ny), 128, smem, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t ww = (int64_t)w * w;
  wgrad_sum_kernel<<<(unsigned)((ww + 255) / 256), 256, 0, s>>>(partial, ny, w, gW);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bias_grad_kernel<<<w, 128, 0, s>>>(dz, N, gb);
  return cudaGetLastError();
}

}  // namespace bsp
