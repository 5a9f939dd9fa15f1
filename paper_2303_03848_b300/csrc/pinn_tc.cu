// pinn_tc.cu -- network evaluation (Section 3.3) with the hidden w x w layers
// on the 5th-generation tensor cores (tcgen05), BF16 operands (kind::f16) or
// TF32 operands (kind::tf32, FP32 values rounded to TF32), FP32 accumulation
// in tensor memory.
//
// One CTA owns a tile of 128 points at a time (the M = 128 rows of every layer
// GEMM) and walks the tiles persistently.  Its warps v, v + 4, ... read the
// same 32 accumulator lanes (points 32 (v % 4) .. + 31) and split the w
// columns of every layer between them: two warps per lane quadrant (256
// threads) up to w = 128, four (512 threads) at w = 256, where the tensor
// memory holds only two CTAs per SM.  Per tile:
//   * input layer (2 or 5 inputs -> w): CUDA cores, FP32, written as the BF16
//     (TF32) A operand of the first square layer;
//   * each square layer h' = tanh(W h + b): one thread issues w/16 (TF32:
//     w/8) tcgen05.mma (M = 128, N = w, K = 16 or 8: 32 bytes of each operand
//     row) into a TMEM accumulator and commits them to an mbarrier; the warps
//     read their 32 lanes back with tcgen05.ld, add the bias, apply FP32 tanh
//     and write the rounded result as the next A operand;
//   * output layer (w -> 1): FP32 tanh of the last hidden layer and a dot
//     product on CUDA cores, the column groups' parts added through shared
//     memory.
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix).  The square layers are packed into that
// layout once per call and fed to shared memory by TMA bulk copies
// (cp.async.bulk) completing on an mbarrier: all layers once, when they fit
// beside several CTAs per SM, else one layer at a time, each copy issued as soon
// as the previous layer's MMAs have completed so that it overlaps the epilogue.
// Every mbarrier wait has a time limit; on expiry the kernel records BS_TIMEOUT
// in a status word, waits (bounded) for its copy in flight, frees its tensor
// memory and returns.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>

#include "bs_internal.h"
#include "tcgen05.cuh"

namespace bsp {

using namespace tc;

// Pack the square layers W_l (l = 2 .. n_lin-1, each w x w) from the FP32
// copy into the core-matrix layout, BF16 or TF32 (rounded with cvt.rna).
template <bool TF>
__global__ void pack_square_kernel(MlpDev m, int w, unsigned char* out) {
  constexpr int EB = TF ? 4 : 2;
  const int n_sq = m.n_lin - 2;
  const int64_t per = (int64_t)w * w;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per * n_sq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / per);
    const int n = (int)((i % per) / w), k = (int)(i % w);
    const float v = m.p32[m.poff[s + 2] + (int64_t)n * w + k];
    unsigned char* dst = out + s * per * EB + canon_off_eb<EB>(n, k, w);
    if constexpr (TF) {
      *reinterpret_cast<uint32_t*>(dst) = to_tf32(v);
    } else {
      *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
    }
  }
}

// Eight FP32 values (columns c .. c + 7 of one operand row) through tanh,
// rounded to the operand type and stored at their core-matrix positions.
template <bool TF>
__device__ __forceinline__ void store_tanh8(unsigned char* sA, int row, int c, int w, const float (&v)[8]) {
  if constexpr (TF) {
    uint4 q0, q1;
    q0.x = to_tf32(tanh_fast(v[0]));
    q0.y = to_tf32(tanh_fast(v[1]));
    q0.z = to_tf32(tanh_fast(v[2]));
    q0.w = to_tf32(tanh_fast(v[3]));
    q1.x = to_tf32(tanh_fast(v[4]));
    q1.y = to_tf32(tanh_fast(v[5]));
    q1.z = to_tf32(tanh_fast(v[6]));
    q1.w = to_tf32(tanh_fast(v[7]));
    *reinterpret_cast<uint4*>(sA + canon_off_eb<4>(row, c, w)) = q0;
    *reinterpret_cast<uint4*>(sA + canon_off_eb<4>(row, c + 4, w)) = q1;
  } else {
    uint4 q;
    q.x = tanh_pack_bf16x2(v[0], v[1]);
    q.y = tanh_pack_bf16x2(v[2], v[3]);
    q.z = tanh_pack_bf16x2(v[4], v[5]);
    q.w = tanh_pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(sA + canon_off(row, c, w)) = q;
  }
}

struct TcArgs {
  MlpDev m;
  const unsigned char* packed;  // square layers, canonical layout, 16-byte aligned
  const double* X;
  int64_t N;
  double* u;
  int w;
  int resident;  // all square layers kept in shared memory
  int* status;   // BS_TIMEOUT recorded here if a wait gave up
};

// First-layer row of a neuron in shared memory: DIN weights, the bias, zeros,
// RW float4s in all (one vector load for 2 inputs, two for 5).
template <int DIN>
constexpr int first_row_f4() { return (DIN + 1 + 3) / 4; }

// NWQ warps share each lane quadrant (its 32 points), w / NWQ columns each:
// 2 (256 threads, up to three CTAs per SM) or, for w = 256, 4 (512 threads and
// two CTAs per SM, the most the tensor memory holds at that width).  TF: TF32
// operands (4 bytes, K = 8 per MMA) instead of BF16 (2 bytes, K = 16).
// TP tiles per CTA: the tiles share each layer's weight copy and its barriers,
// each with its own operand buffer and accumulator (see tc_tiles_per_cta).
template <int DIN, int NWQ, bool TF, int TP>
__global__ void __launch_bounds__(128 * NWQ * TP, NWQ * TP == 4 ? 2 : 0) mlp_tc_kernel(TcArgs a) {
  static_assert(DIN == 2 || DIN == 5, "2 or 5 inputs");
  constexpr int RW = first_row_f4<DIN>();
  constexpr int EB = TF ? 4 : 2;       // operand bytes
  constexpr int KPM = 32 / EB;         // K of one MMA
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int w = a.w, t = threadIdx.x, warp = t >> 5;
  const int ts = warp / (4 * NWQ), wt = warp % (4 * NWQ);  // tile slot, warp within the tile's warps
  const int pt = (wt & 3) * 32 + (t & 31);  // this thread's point (accumulator lane)
  const int hw = w / NWQ, cb = (wt >> 2) * hw;  // and its columns [cb, cb + hw)
  const int n_sq = m.n_lin - 2;
  const uint32_t wbytes = (uint32_t)w * w * EB;
  // shared memory carve-up
  unsigned char* sW = smem;                                             // n_sq (resident) or 1 square layer
  unsigned char* sA0 = sW + (a.resident ? (size_t)n_sq : 1) * wbytes;   // TP x (128 x w operand)
  unsigned char* sA = sA0 + (size_t)ts * 128 * w * EB;                   // this thread's tile
  float* sW1 = reinterpret_cast<float*>(sA0 + (size_t)TP * 128 * w * EB);  // w rows of RW float4 (W_1, b_1)
  float* sB = sW1 + w * 4 * RW;                                         // biases of hidden layers, (n_lin-1) x w
  float* sWo = sB + (m.n_lin - 1) * w;                                  // output weights, w
  uint64_t* bar = reinterpret_cast<uint64_t*>(sWo + w + 2);             // [0] MMA done, [1] weights landed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  __shared__ int s_fail;
  __shared__ float s_dot[2][TP][NWQ - 1][128];  // output partial sums of the other column groups, by tile parity

  // parameters into shared memory; the input map to [-1, 1] in FP32 registers
  for (int i = t; i < w * 4 * RW; i += blockDim.x) {
    const int o = i / (4 * RW), k = i % (4 * RW);
    sW1[i] = k < DIN ? m.p32[m.poff[1] + o * DIN + k] : (k == DIN ? m.p32[m.poff[1] + w * DIN + o] : 0.0f);
  }
  for (int l = 1; l < m.n_lin; ++l)
    for (int o = t; o < w; o += blockDim.x)
      sB[(l - 1) * w + o] = m.p32[m.poff[l] + (int64_t)w * m.widths[l - 1] + o];
  for (int o = t; o < w; o += blockDim.x) sWo[o] = m.p32[m.poff[m.n_lin] + o];
  const float bout = m.p32[m.poff[m.n_lin] + w];
  float sc[DIN], of[DIN];
#pragma unroll
  for (int i = 0; i < DIN; ++i) {
    const double s = 2.0 / (m.hi[i] - m.lo[i]);
    sc[i] = (float)s;
    of[i] = (float)(-s * m.lo[i] - 1.0);
  }
  const int64_t ntiles = (a.N + 127) / 128, ngroups = (ntiles + TP - 1) / TP;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // first weight copy: every layer (resident) or layer 0
  bool w_pending = false;  // thread 0: a weight copy is in flight
  uint32_t ph_w = 0, ph_mma = 0;
  if (t == 0 && n_sq > 0 && (int64_t)blockIdx.x < ngroups) {
    bulk_load(sW, a.packed, a.resident ? (uint32_t)n_sq * wbytes : wbytes, &bar[1]);
    w_pending = true;
  }
  // tensor memory: w FP32 columns x 128 lanes per tile
  uint32_t ncols = 32;
  while ((int)ncols < w) ncols <<= 1;
  const uint32_t nalloc = ncols * TP;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(nalloc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = TF ? make_idesc_tf32(w) : make_idesc_bf16(w);
  const uint32_t sbo = (uint32_t)(w * EB / 16) * 128;  // next 8-row group

  // this warp's accumulator lanes in its tile's columns
  const uint32_t tl = tmem + (uint32_t)ts * ncols + ((uint32_t)((wt & 3) * 32) << 16);
  double xn[DIN];  // inputs of this thread's point in the next tile (prefetched)
  {
    const int64_t p = ((int64_t)blockIdx.x * TP + ts) * 128 + pt;
#pragma unroll
    for (int i = 0; i < DIN; ++i) xn[i] = p < a.N ? a.X[p * DIN + i] : 0.0;
  }
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const int64_t tile = grp * TP + ts;
    const int64_t p = tile * 128 + pt;
    const bool valid = p < a.N;
    const bool last_tile = grp + gridDim.x >= ngroups;
    float xh[DIN];
#pragma unroll
    for (int i = 0; i < DIN; ++i) xh[i] = fmaf((float)xn[i], sc[i], of[i]);
    if (!last_tile) {
      const int64_t q = p + (int64_t)gridDim.x * TP * 128;
#pragma unroll
      for (int i = 0; i < DIN; ++i) xn[i] = q < a.N ? a.X[q * DIN + i] : 0.0;
    }
    // input layer on CUDA cores
    float dot = 0.0f;  // output accumulator (used here when there is no square layer)
    for (int o0 = cb; o0 < cb + hw; o0 += 16) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int ob = o0 + half * 8;
        float z[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4* row = reinterpret_cast<const float4*>(sW1) + (ob + j) * RW;
          const float4 r0 = row[0];
          if constexpr (DIN == 2) {
            z[j] = fmaf(r0.y, xh[1], fmaf(r0.x, xh[0], r0.z));
          } else {
            const float4 r1 = row[1];
            z[j] = fmaf(r1.x, xh[4], fmaf(r0.w, xh[3], fmaf(r0.z, xh[2], fmaf(r0.y, xh[1], fmaf(r0.x, xh[0], r1.y)))));
          }
        }
        if (n_sq == 0) {
#pragma unroll
          for (int j = 0; j < 8; ++j) dot = fmaf(sWo[ob + j], tanh_fast(z[j]), dot);
        } else {
          store_tanh8<TF>(sA, pt, ob, w, z);
        }
      }
    }
    // square layers on the tensor cores
    for (int s = 0; s < n_sq; ++s) {
      const unsigned char* wl = sW + (a.resident ? (size_t)s * wbytes : 0);
      if (t == 0 && w_pending) {  // the weights of this layer have landed
        if (mbar_wait_bounded(&bar[1], ph_w)) {
          ph_w ^= 1u;
          w_pending = false;
        } else {
          s_fail = 1;
        }
      }
      fence_proxy_async();  // generic-proxy writes of A visible to the tensor core
      fence_before();
      __syncthreads();
      fence_after();
      if (s_fail) break;
      if (t == 0) {
        const uint32_t bb = smem_u32(wl);
#pragma unroll
        for (int q = 0; q < TP; ++q) {  // every tile of the group against the same weights
          const uint32_t aa = smem_u32(sA0) + (uint32_t)q * 128 * w * EB, dq = tmem + (uint32_t)q * ncols;
          for (int kk = 0; kk < w / KPM; ++kk) {  // each MMA: 2 core matrices (32 bytes) along K
            const uint64_t da = make_desc(aa + kk * 256, 128, sbo);
            const uint64_t db = make_desc(bb + kk * 256, 128, sbo);
            if constexpr (TF) {
              mma_tf32(dq, da, db, idesc, kk > 0 ? 1u : 0u);
            } else {
              mma_bf16(dq, da, db, idesc, kk > 0 ? 1u : 0u);
            }
          }
        }
        mma_commit(&bar[0]);
      }
      // thread 0 waits for the MMAs (the others wait at the barrier without
      // taking issue slots from the other CTAs' epilogues), then the
      // tcgen05 fences order the accumulator reads after it
      if (t == 0) {
        if (!mbar_wait_bounded(&bar[0], ph_mma)) {
          s_fail = 1;
        } else if (!a.resident && !(last_tile && s == n_sq - 1)) {
          // the MMAs have read this layer's weights: fetch the next layer's while
          // the epilogue runs (one layer at a time when they are not resident)
          const int nxt = s + 1 < n_sq ? s + 1 : 0;
          bulk_load(sW, a.packed + (size_t)nxt * wbytes, wbytes, &bar[1]);
          w_pending = true;
        }
      }
      ph_mma ^= 1u;
      fence_before();
      __syncthreads();
      fence_after();
      if (s_fail) break;
      // epilogue: TMEM -> registers (warp reads its 32 lanes), bias, tanh
      const bool last = s == n_sq - 1;
      const float* bl = sB + (s + 1) * w;
      for (int c = cb; c < cb + hw; c += 16) {
        uint32_t r[16];
        tmem_ld16_nowait(tl + (uint32_t)c, r);
        tmem_wait_ld();
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 bq = *reinterpret_cast<const float4*>(bl + c + j);
          v[j] = __uint_as_float(r[j]) + bq.x;
          v[j + 1] = __uint_as_float(r[j + 1]) + bq.y;
          v[j + 2] = __uint_as_float(r[j + 2]) + bq.z;
          v[j + 3] = __uint_as_float(r[j + 3]) + bq.w;
        }
        if (last) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) {
            const float4 wq = *reinterpret_cast<const float4*>(sWo + c + j);
            dot = fmaf(wq.x, tanh_fast(v[j]), dot);
            dot = fmaf(wq.y, tanh_fast(v[j + 1]), dot);
            dot = fmaf(wq.z, tanh_fast(v[j + 2]), dot);
            dot = fmaf(wq.w, tanh_fast(v[j + 3]), dot);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; j += 8) {
            const float (&v8)[8] = *reinterpret_cast<const float(*)[8]>(v + j);
            store_tanh8<TF>(sA, pt, c + j, w, v8);
          }
        }
      }
      fence_before();  // tensor-memory reads done before the next MMA overwrites the accumulator
    }
    if (s_fail) break;
    // the two column halves of the output dot product (two buffers: without a
    // square layer this is the only barrier of a tile)
    const int par = (int)((grp / gridDim.x) & 1);
    if (wt >= 4) s_dot[par][ts][(wt >> 2) - 1][pt] = dot;
    __syncthreads();
    if (wt < 4 && valid) {
      float u = dot;
#pragma unroll
      for (int q = 0; q < NWQ - 1; ++q) u += s_dot[par][ts][q][pt];
      a.u[p] = (double)(u + bout);
    }
  }
  // a weight copy still in flight (only after a failed wait) lands before exit
  if (t == 0 && w_pending) (void)mbar_wait_bounded(&bar[1], ph_w);
  fence_before();
  __syncthreads();
  fence_after();
  if (s_fail && t == 0) atomicExch(a.status, 6);  // BS_TIMEOUT
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nalloc) : "memory");
  }
}

// One bounded wait as the network kernels do it, on a barrier that one thread
// completes (arrive != 0) or that nothing completes: status = BS_OK or BS_TIMEOUT.
__global__ void wait_probe_kernel(int arrive, long long limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
  const bool ok = mbar_wait_bounded(&bar, 0u, limit);
  __syncthreads();
  if (threadIdx.x == 0) *status = ok ? 0 : 6;  // BS_OK, BS_TIMEOUT
}

cudaError_t launch_wait_probe(int arrive, long long limit, int* status, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(arrive, limit, status);
  return cudaGetLastError();
}

// Shape supported by the tensor-core path: all hidden layers w x w (w a multiple
// of 32, 32 <= w <= 256), 2 or 5 inputs, output width 1.
bool tc_supported(const MlpDev& m) {
  if (m.n_lin < 2 || !(m.d_in == 2 || m.d_in == 5)) return false;
  const int w = m.widths[1];
  if (w < 32 || w > 256 || (w % 32) != 0) return false;
  for (int l = 1; l < m.n_lin; ++l)
    if (m.widths[l] != w) return false;
  return m.widths[m.n_lin] == 1;
}

// Tiles per CTA of the tensor-core kernel: two for TF32 up to w = 128, where
// the 4-byte operands leave room for one CTA per SM and the second tile doubles
// the work in flight (1.44e9 -> 1.74e9 points/s on 5->6x128); one for BF16,
// whose three independent one-tile CTAs per SM overlap one another's GEMMs and
// epilogues better than two CTAs of two tiles in step (115.6 against 123.5 ms
// for the batched workload's table); one at w = 256.
static int tc_tiles_per_cta(int w, int eb) { return (eb == 4 && w <= 128) ? 2 : 1; }

// Shared memory of the tensor-core kernel: square-layer weights (all layers
// when that still leaves room for several CTAs per SM, else one), the 128 x w
// activation operand of each tile, the FP32 input/output layers and biases,
// two mbarriers.  eb: operand bytes (2 BF16, 4 TF32).
static size_t tc_smem_bytes(const MlpDev& m, int* resident, int eb) {
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  const size_t wbytes = (size_t)w * w * eb;
  const size_t rw = m.d_in == 2 ? first_row_f4<2>() : first_row_f4<5>();
  const size_t fixed = (size_t)tc_tiles_per_cta(w, eb) * 128 * w * eb +
                       sizeof(float) * ((size_t)w * 4 * rw + (size_t)(m.n_lin - 1) * w + w + 2) + 32 + 1024;
  const int res = (n_sq > 0 && (size_t)n_sq * wbytes + fixed <= 96 * 1024) ? 1 : 0;
  if (resident) *resident = res;
  return (res ? (size_t)n_sq : 1) * wbytes + fixed;
}

bool tc_fits(const MlpDev& m, bool tf32) {
  return tc_supported(m) && tc_smem_bytes(m, nullptr, tf32 ? 4 : 2) <= 220 * 1024;
}

// Room for the square layers in either operand type (TF32: 4 bytes each).
size_t tc_packed_bytes(const MlpDev& m) {
  const int w = m.widths[1];
  const int n_sq = m.n_lin - 2;
  return (size_t)(n_sq > 0 ? n_sq : 0) * w * w * 4;
}

cudaError_t launch_mlp_eval_tc(const MlpDev& m, unsigned char* packed, const double* X, int64_t N, double* u,
                               int* status, cudaStream_t s, bool tf32) {
  if (N <= 0) return cudaSuccess;
  if (((uintptr_t)packed & 15) != 0) return cudaErrorInvalidValue;  // TMA source alignment
  const int w = m.widths[1], n_sq = m.n_lin - 2;
  cudaError_t e = cudaSuccess;
  if (n_sq > 0) {
    if (tf32) {
      pack_square_kernel<true><<<148, 256, 0, s>>>(m, w, packed);
    } else {
      pack_square_kernel<false><<<148, 256, 0, s>>>(m, w, packed);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int resident = 0;
  const size_t smem = tc_smem_bytes(m, &resident, tf32 ? 4 : 2);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  TcArgs a{m, packed, X, N, u, w, resident, status};
  const bool wide = w == 256;  // four warps per lane quadrant, one tile per CTA
  const int tp = tc_tiles_per_cta(w, tf32 ? 4 : 2);
  const int threads = wide ? 512 : 256 * tp;
  auto kern = tf32 ? (m.d_in == 2 ? (wide ? mlp_tc_kernel<2, 4, true, 1> : mlp_tc_kernel<2, 2, true, 2>)
                                  : (wide ? mlp_tc_kernel<5, 4, true, 1> : mlp_tc_kernel<5, 2, true, 2>))
                   : (m.d_in == 2 ? (wide ? mlp_tc_kernel<2, 4, false, 1> : mlp_tc_kernel<2, 2, false, 1>)
                                  : (wide ? mlp_tc_kernel<5, 4, false, 1> : mlp_tc_kernel<5, 2, false, 1>));
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  // CTAs per SM from the shared memory each one takes (dynamic + static + the
  // per-block reservation) with the carveout at its maximum, and the registers
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  int dev = 0, nsm = 148, sm_smem = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  int per_sm = (int)((size_t)sm_smem / (smem + fa.sharedSizeBytes + (size_t)reserved));
  const int by_regs = 65536 / (threads * (fa.numRegs > 0 ? fa.numRegs : 255));
  if (per_sm > by_regs) per_sm = by_regs;
  if (per_sm < 1) per_sm = 1;
  int ncols = 32;
  while (ncols < w) ncols <<= 1;
  if (per_sm > 512 / (ncols * tp)) per_sm = 512 / (ncols * tp);  // tensor memory: 512 columns per SM
  if (per_sm > 4) per_sm = 4;
  const int64_t ngroups = ((N + 127) / 128 + tp - 1) / tp;
  const int64_t grid = ngroups < (int64_t)nsm * per_sm ? ngroups : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bsp
