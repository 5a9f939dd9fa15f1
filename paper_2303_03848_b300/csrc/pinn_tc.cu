// pinn_tc.cu -- network evaluation (Section 3.3) with the hidden w x w layers
// on the 5th-generation tensor cores (tcgen05), BF16 or TF32 operands, FP32
// accumulation in tensor memory.
//
// One CTA of 128 threads owns a tile of 128 points (the M = 128 rows of every
// layer GEMM, thread t = point t = TMEM lane t).  Per tile:
//   * input layer (2 or 5 inputs -> w): CUDA cores, FP32, tanh, written as
//     the A operand of the first square layer;
//   * each square layer h' = tanh(W h + b): one thread issues w/K tcgen05.mma
//     (M = 128, N = w, K = 16 for BF16 / 8 for TF32) into a TMEM accumulator and
//     commits them to an mbarrier; the four warps read their 32 lanes back with
//     tcgen05.ld, add the bias, apply tanh and write the next A operand;
//   * output layer (w -> 1): a dot product on CUDA cores.
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix); the weights are packed into that layout
// once per call and stay resident for all tiles when they fit.
// Every wait on the mbarrier has an iteration limit; on expiry the kernel
// records BS_TIMEOUT in a status word, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>

#include "bs_internal.h"

namespace bsp {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared memory matrix descriptor: no swizzle, K-major.  LBO = byte distance of
// core matrices adjacent along K, SBO = along M/N; descriptor version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: D FP32, A/B format (1 BF16 for kind::f16, 2 TF32 for
// kind::tf32), both K-major, N = n, M = 128.
__device__ __forceinline__ uint32_t make_idesc(int fmt, int n) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (TF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok;
}

// Bounded wait: true when the phase completed, false after the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1LL << 33)) return false;  // about 4 s at 2 GHz
  }
  return true;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element (row, k) in an R x K K-major no-swizzle operand with
// element size E (16/E elements per core-matrix row).
__host__ __device__ __forceinline__ uint32_t canon_off(int row, int k, int K, int E) {
  const int kpc = 16 / E;
  return (uint32_t)(((row >> 3) * (K / kpc) + k / kpc) * 128 + (row & 7) * 16 + (k % kpc) * E);
}

}  // namespace

// Pack the square layers W_l (l = 2 .. n_lin-1, each w x w) from the FP32
// copy into the core-matrix layout, BF16 or TF32-rounded FP32.
__global__ void pack_square_kernel(MlpDev m, int w, int tf32, unsigned char* out) {
  const int n_sq = m.n_lin - 2;
  const int E = tf32 ? 4 : 2;
  const int64_t per = (int64_t)w * w;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < per * n_sq;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / per);
    const int n = (int)((i % per) / w), k = (int)(i % w);
    const float v = m.p32[m.poff[s + 2] + (int64_t)n * w + k];
    unsigned char* dst = out + s * per * E + canon_off(n, k, w, E);
    if (tf32) {
      *reinterpret_cast<float*>(dst) = to_tf32(v);
    } else {
      *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
    }
  }
}

struct TcArgs {
  MlpDev m;
  const unsigned char* packed;  // square layers, canonical layout
  const double* X;
  int64_t N;
  double* u;
  int w;
  int resident;  // all square layers kept in shared memory
  int* status;   // BS_TIMEOUT recorded here if a wait gave up
};

template <bool TF32, int DIN>
__global__ void __launch_bounds__(128) mlp_tc_kernel(TcArgs a) {
  constexpr int E = TF32 ? 4 : 2;
  constexpr int KSTEP = TF32 ? 8 : 16;  // K of one MMA
  extern __shared__ __align__(1024) unsigned char smem[];
  const MlpDev& m = a.m;
  const int w = a.w, t = threadIdx.x, warp = t >> 5;
  const int n_sq = m.n_lin - 2;
  constexpr int d_in = DIN;  // 2 or 5 inputs
  const uint32_t wbytes = (uint32_t)w * w * E;
  // shared memory carve-up
  unsigned char* sW = smem;                                       // n_sq (resident) or 1 square layer
  unsigned char* sA = sW + (a.resident ? (size_t)n_sq : 1) * wbytes;  // 128 x w operand
  float* sW1 = reinterpret_cast<float*>(sA + (size_t)128 * w * E);    // w x d_in
  float* sB = sW1 + w * d_in;                                     // biases of hidden layers, (n_lin-1) x w
  float* sWo = sB + (m.n_lin - 1) * w;                            // output weights, w
  uint64_t* bar = reinterpret_cast<uint64_t*>(sWo + w + 2);       // 8-byte aligned (w even)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  __shared__ int s_fail;

  // parameters into shared memory
  for (int i = t; i < w * d_in; i += 128) sW1[i] = m.p32[m.poff[1] + i];
  for (int l = 1; l < m.n_lin; ++l)
    for (int o = t; o < w; o += 128) sB[(l - 1) * w + o] = m.p32[m.poff[l] + (int64_t)w * m.widths[l - 1] + o];
  for (int o = t; o < w; o += 128) sWo[o] = m.p32[m.poff[m.n_lin] + o];
  const float bout = m.p32[m.poff[m.n_lin] + w];
  if (a.resident) {
    const uint4* src = reinterpret_cast<const uint4*>(a.packed);
    uint4* dst = reinterpret_cast<uint4*>(sW);
    for (size_t i = t; i < (size_t)n_sq * wbytes / 16; i += 128) dst[i] = src[i];
  }
  if (t == 0) {
    mbar_init(bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tensor memory: w FP32 columns x 128 lanes
  uint32_t ncols = 32;
  while ((int)ncols < w) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc(TF32 ? 2 : 1, w);
  const uint32_t sbo = (uint32_t)(w / (16 / E)) * 128;  // next 8-row group
  uint32_t phase = 0;
  const int64_t ntiles = (a.N + 127) / 128;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t p = tile * 128 + t;
    const bool valid = p < a.N;
    // input layer on CUDA cores
    float xh[DIN];
#pragma unroll
    for (int i = 0; i < d_in; ++i) {
      const double x = valid ? a.X[p * d_in + i] : 0.0;
      xh[i] = (float)(2.0 / (m.hi[i] - m.lo[i]) * (x - m.lo[i]) - 1.0);
    }
    float dot = 0.0f;  // output layer accumulator (used when the last hidden layer is computed here)
    for (int o0 = 0; o0 < w; o0 += 16 / E * 2) {
      // one 16-byte store per core-matrix row chunk (8 BF16 or 4 TF32 values), two chunks per iteration
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int ob = o0 + half * (16 / E);
        float hv[8];
#pragma unroll
        for (int j = 0; j < 16 / E; ++j) {
          float z = sB[ob + j];
#pragma unroll
          for (int i = 0; i < d_in; ++i) z = fmaf(sW1[(ob + j) * d_in + i], xh[i], z);
          hv[j] = tanh_fast(z);
        }
        if (n_sq == 0) {
#pragma unroll
          for (int j = 0; j < 16 / E; ++j) dot = fmaf(sWo[ob + j], hv[j], dot);
        } else if (TF32) {
          float4 q = make_float4(to_tf32(hv[0]), to_tf32(hv[1]), to_tf32(hv[2]), to_tf32(hv[3]));
          *reinterpret_cast<float4*>(sA + canon_off(t, ob, w, E)) = q;
        } else {
          __nv_bfloat162 q0 = __floats2bfloat162_rn(hv[0], hv[1]), q1 = __floats2bfloat162_rn(hv[2], hv[3]),
                          q2 = __floats2bfloat162_rn(hv[4], hv[5]), q3 = __floats2bfloat162_rn(hv[6], hv[7]);
          uint4 q;
          q.x = *reinterpret_cast<uint32_t*>(&q0);
          q.y = *reinterpret_cast<uint32_t*>(&q1);
          q.z = *reinterpret_cast<uint32_t*>(&q2);
          q.w = *reinterpret_cast<uint32_t*>(&q3);
          *reinterpret_cast<uint4*>(sA + canon_off(t, ob, w, E)) = q;
        }
      }
    }
    // square layers on the tensor cores
    for (int s = 0; s < n_sq; ++s) {
      const unsigned char* wl = sW + (a.resident ? (size_t)s * wbytes : 0);
      if (!a.resident) {
        const uint4* src = reinterpret_cast<const uint4*>(a.packed + (size_t)s * wbytes);
        uint4* dst = reinterpret_cast<uint4*>(sW);
        for (uint32_t i = t; i < wbytes / 16; i += 128) dst[i] = src[i];
      }
      fence_proxy_async();  // generic-proxy writes of A (and W) visible to the tensor core
      fence_before();
      __syncthreads();
      fence_after();
      if (t == 0) {
        const uint32_t aa = smem_u32(sA), bb = smem_u32(wl);
        for (int kk = 0; kk < w / KSTEP; ++kk) {
          const uint64_t da = make_desc(aa + kk * 256, 128, sbo);
          const uint64_t db = make_desc(bb + kk * 256, 128, sbo);
          mma<TF32>(tmem, da, db, idesc, kk > 0 ? 1u : 0u);
        }
        mma_commit(bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase);
      phase ^= 1;
      if (!ok) s_fail = 1;
      fence_after();
      __syncthreads();
      if (s_fail) break;
      // epilogue: TMEM -> registers (warp reads its 32 lanes), bias, tanh
      const bool last = s == n_sq - 1;
      const float* bl = sB + (s + 1) * w;
      for (int c = 0; c < w; c += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 bq = *reinterpret_cast<const float4*>(bl + c + j);
          v[j] = tanh_fast(v[j] + bq.x);
          v[j + 1] = tanh_fast(v[j + 1] + bq.y);
          v[j + 2] = tanh_fast(v[j + 2] + bq.z);
          v[j + 3] = tanh_fast(v[j + 3] + bq.w);
        }
        if (last) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 wq = *reinterpret_cast<const float4*>(sWo + c + j);
            dot = fmaf(wq.x, v[j], dot);
            dot = fmaf(wq.y, v[j + 1], dot);
            dot = fmaf(wq.z, v[j + 2], dot);
            dot = fmaf(wq.w, v[j + 3], dot);
          }
        } else if (TF32) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            float4 q = make_float4(to_tf32(v[j]), to_tf32(v[j + 1]), to_tf32(v[j + 2]), to_tf32(v[j + 3]));
            *reinterpret_cast<float4*>(sA + canon_off(t, c + j, w, E)) = q;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; j += 8) {
            __nv_bfloat162 q0 = __floats2bfloat162_rn(v[j], v[j + 1]), q1 = __floats2bfloat162_rn(v[j + 2], v[j + 3]),
                            q2 = __floats2bfloat162_rn(v[j + 4], v[j + 5]),
                            q3 = __floats2bfloat162_rn(v[j + 6], v[j + 7]);
            uint4 q;
            q.x = *reinterpret_cast<uint32_t*>(&q0);
            q.y = *reinterpret_cast<uint32_t*>(&q1);
            q.z = *reinterpret_cast<uint32_t*>(&q2);
            q.w = *reinterpret_cast<uint32_t*>(&q3);
            *reinterpret_cast<uint4*>(sA + canon_off(t, c + j, w, E)) = q;
          }
        }
      }
      fence_before();  // tensor-memory reads done before the next MMA overwrites the accumulator
    }
    if (s_fail) break;
    if (valid) a.u[p] = (double)(dot + bout);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (s_fail && t == 0) atomicExch(a.status, 6);  // BS_TIMEOUT
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
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

// Shared memory of the tensor-core kernel: square-layer weights (all layers
// when they fit in 200 KB, else one), the 128 x w activation operand, the FP32
// input/output layers and biases.
static size_t tc_smem_bytes(const MlpDev& m, int tf32, int* resident) {
  const int w = m.widths[1], n_sq = m.n_lin - 2, E = tf32 ? 4 : 2;
  const size_t wbytes = (size_t)w * w * E;
  const size_t fixed = (size_t)128 * w * E +
                       sizeof(float) * ((size_t)w * m.d_in + (size_t)(m.n_lin - 1) * w + w + 2) + 16 + 1024;
  // resident only while it still leaves room for several CTAs per SM (latency
  // hiding); otherwise each layer is reloaded from L2 per tile
  const int res = (n_sq > 0 && (size_t)n_sq * wbytes + fixed <= 96 * 1024) ? 1 : 0;
  if (resident) *resident = res;
  return (res ? (size_t)n_sq : 1) * wbytes + fixed;
}

bool tc_fits(const MlpDev& m, int tf32) { return tc_supported(m) && tc_smem_bytes(m, tf32, nullptr) <= 220 * 1024; }

size_t tc_packed_bytes(const MlpDev& m, int tf32) {
  const int w = m.widths[1];
  const int n_sq = m.n_lin - 2;
  return (size_t)(n_sq > 0 ? n_sq : 0) * w * w * (tf32 ? 4 : 2);
}

cudaError_t launch_mlp_eval_tc(const MlpDev& m, int tf32, unsigned char* packed, const double* X, int64_t N,
                               double* u, int* status, cudaStream_t s) {
  if (N <= 0) return cudaSuccess;
  const int w = m.widths[1], n_sq = m.n_lin - 2, E = tf32 ? 4 : 2;
  cudaError_t e = cudaSuccess;
  if (n_sq > 0) {
    pack_square_kernel<<<148, 256, 0, s>>>(m, w, tf32, packed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  (void)E;
  int resident = 0;
  const size_t smem = tc_smem_bytes(m, tf32, &resident);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  TcArgs a{m, packed, X, N, u, w, resident, status};
  auto kern = tf32 ? (m.d_in == 2 ? mlp_tc_kernel<true, 2> : mlp_tc_kernel<true, 5>)
                   : (m.d_in == 2 ? mlp_tc_kernel<false, 2> : mlp_tc_kernel<false, 5>);
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  // CTAs per SM from the shared memory each one takes (dynamic + static + the
  // per-block reservation) with the carveout at its maximum; the registers
  // (128 threads x <= 255) never limit below 2
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
  int dev = 0, nsm = 148, sm_smem = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  int per_sm = (int)((size_t)sm_smem / (smem + fa.sharedSizeBytes + (size_t)reserved));
  const int by_regs = 65536 / (128 * (fa.numRegs > 0 ? fa.numRegs : 255));
  if (per_sm > by_regs) per_sm = by_regs;
  if (per_sm < 1) per_sm = 1;
  int ncols = 32;
  while (ncols < w) ncols <<= 1;
  if (per_sm > 512 / ncols) per_sm = 512 / ncols;  // tensor memory: 512 columns per SM
  if (per_sm > 4) per_sm = 4;
  const int64_t ntiles = (N + 127) / 128;
  const int64_t grid = ntiles < (int64_t)nsm * per_sm ? ntiles : (int64_t)nsm * per_sm;
  kern<<<(unsigned)grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bsp
