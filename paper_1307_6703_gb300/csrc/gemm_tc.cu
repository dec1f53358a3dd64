// gemm_tc.cu -- the network's matrix products (include/fno.h) on the
// fifth-generation tensor cores of sm_103a: BF16 operands staged in shared
// memory by TMA, tcgen05.mma issued by one thread, FP32 accumulators in
// tensor memory read back with tcgen05.ld; plus a plain FP32 SIMT product
// for the full-precision mode of the network.
//
// BF16 product (gemm_tn_bf16):  D[b](m, n) = sum_k X[b](m, k) Y[b](n, k)
// with X and Y row-major in k (k contiguous, "K-major" for both operands),
// written to C[b] at c + b * sC + m * cm + n * cn as C = D + beta * C.  A
// CTA computes a 128 x BN tile of D (one M = 128, N = BN MMA shape) over a
// K range, 64 columns of K per pipeline stage: one TMA box of 128 x 64 of X
// and one of BN x 64 of Y per stage, both 128-byte swizzled (a row of 64
// BF16 is one 128-byte swizzle row, eight rows one 1024-byte swizzle atom),
// four stages in flight (one when the K range fits a single stage).  Thread 0 requests the boxes and issues the four
// K = 16 MMAs of a stage; their completion (tcgen05.commit) frees the stage.
// The four warps then read the accumulator rows 32w .. 32w + 31 of tensor
// memory and store them.  Rows, columns and K beyond the operands are
// zero-filled by TMA and not stored.  Every wait is bounded: on give-up the
// kernel sets *err, waits (bounded) for its copies in flight, frees its
// tensor memory and returns.
//
// ksplit > 1 splits K: batch index bz = b * ksplit + s covers
// k in [s * kper, (s + 1) * kper) and writes its own output slice bz (the
// caller adds the slices).
#include <algorithm>
#include <cstdint>
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fno.h"
#include "gemm_tc.h"

namespace tc {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Shared-memory matrix descriptor of a K-major, 128-byte swizzled operand
// tile (tcgen05 format): start address >> 4 in bits 0-13, leading byte
// offset (unused for swizzled K-major operands) 0, stride byte offset
// (between 8-row groups: 1024 bytes) >> 4 in bits 32-45, descriptor version
// 1 in bits 46-47, swizzle mode 128 B (2) in bits 61-63.
__device__ __forceinline__ uint64_t kmajor_sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1, the same type for both), both K-major (bits 15,
// 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// Stages: 1 when the K range fits one stage (no pipeline to keep full, and
// a small footprint lets more CTAs share an SM), else 4.
template <int BN, int kStages>
struct __align__(1024) Smem {
  __nv_bfloat16 a[kStages][kBM * kBK];  // 16 KB per stage
  __nv_bfloat16 b[kStages][BN * kBK];   // BN * 128 bytes per stage
  unsigned long long full[kStages], empty[kStages], done;
  uint32_t tmem;
  static_assert(sizeof(a) + sizeof(b) >= 4 * 32 * 33 * sizeof(float), "the epilogue's staging tiles reuse stage memory");
};

__device__ __forceinline__ void tma_load_3d(const CUtensorMap *map, uint32_t dst, uint32_t bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

template <int BN, int kStages>
__global__ void __launch_bounds__(kThreads)
gemm_tn_bf16_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap my,
                    const GemmParams p) {
  extern __shared__ unsigned char raw[];
  // the swizzled tiles need 1024-byte alignment
  using Sm = Smem<BN, kStages>;
  Sm &S = *reinterpret_cast<Sm *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int mt = blockIdx.x, nt = blockIdx.y, bz = blockIdx.z;
  const int b = bz / p.ksplit, ks = bz - b * p.ksplit;
  const int k0 = ks * p.kper, k1 = min(p.K, k0 + p.kper);
  const int nk = k1 > k0 ? (k1 - k0 + kBK - 1) / kBK : 0;
  constexpr uint32_t kTx = (uint32_t)(kBM + BN) * kBK * 2;

  if (t == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.empty[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // BN FP32 columns of tensor memory for the accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;

  bool ok = true;
  if (t == 0) {
    const int xz = p.x_batched ? b : 0, yz = p.y_batched ? b : 0;
    auto load = [&](int c) {
      const int s = c % kStages;
      const uint32_t bar = smem_u32(&S.full[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kTx) : "memory");
      tma_load_3d(&mx, smem_u32(S.a[s]), bar, k0 + c * kBK, mt * kBM, xz);
      tma_load_3d(&my, smem_u32(S.b[s]), bar, k0 + c * kBK, nt * BN, yz);
    };
    int issued = 0;
    for (; issued < min(kStages, nk); ++issued) load(issued);
    constexpr uint32_t idesc = idesc_bf16<BN>();
    for (int c = 0; c < nk && ok; ++c) {
      const int s = c % kStages;
      if (!mbar_try(smem_u32(&S.full[s]), (uint32_t)((c / kStages) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(S.a[s]), b0 = smem_u32(S.b[s]);
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j) {  // K = 16 per MMA: 32 bytes along the swizzle row
        const uint64_t ad = kmajor_sw128_desc(a0 + 32 * j), bd = kmajor_sw128_desc(b0 + 32 * j);
        const uint32_t acc = (c > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      // the stage is free once these MMAs have read it
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&S.empty[s]))
                   : "memory");
      // refill the stage of the previous chunk (its MMAs were queued one
      // chunk earlier, so the tensor core still has this chunk's work)
      if (c >= 1 && c - 1 + kStages < nk) {
        const int pc = c - 1, ps = pc % kStages;
        if (!mbar_try(smem_u32(&S.empty[ps]), (uint32_t)((pc / kStages) & 1))) {
          ok = false;
          break;
        }
        load(pc + kStages);
        ++issued;
      }
    }
    if (!ok) {
      atomicOr(p.err, 1);
      // every copy still in flight lands before the CTA leaves
      for (int c = max(0, issued - kStages); c < issued; ++c)
        (void)mbar_try(smem_u32(&S.full[c % kStages]), (uint32_t)((c / kStages) & 1));
    }
    // all MMAs issued so far complete -> done
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&S.done))
                 : "memory");
  }
  __syncthreads();
  const bool done_ok = mbar_try(smem_u32(&S.done), 0u);
  if (!done_ok && lane == 0) atomicOr(p.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // Epilogue: warp w holds accumulator rows 32w .. 32w + 31 (one per lane),
  // read 32 columns at a time.  Where n is the output's contiguous index
  // (cn == 1) each 32 x 32 block goes through a per-warp shared tile so that
  // a store instruction writes 32 consecutive n of one row; otherwise lanes
  // (consecutive m) already write consecutive addresses.
  const int m = mt * kBM + warp * 32 + lane;
  float *crow = p.c + (long long)bz * p.sC + (long long)m * p.cm;
  const bool row_major = p.cn == 1;
  float *tile = reinterpret_cast<float *>(&S.a[0][0]) + warp * 32 * 33;  // stages are no longer read
  const bool valid = ok && done_ok;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (!valid) continue;
    const int nb = nt * BN + c0;
    if (row_major) {
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = nk > 0 ? __uint_as_float(r[j]) : 0.f;
      __syncwarp();
      const int n = nb + lane;
      float *base = p.c + (long long)bz * p.sC + (long long)(mt * kBM + warp * 32) * p.cm + n;
      const int rows = min(32, p.M - (mt * kBM + warp * 32));
      if (p.beta != 0.f) {  // all old values first: the loads must not wait for the stores
        float old[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) old[i] = (i < rows && n < p.N) ? base[(long long)i * p.cm] : 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < rows && n < p.N) base[(long long)i * p.cm] = fmaf(p.beta, old[i], tile[i * 33 + lane]);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < rows && n < p.N) base[(long long)i * p.cm] = tile[i * 33 + lane];
      }
      __syncwarp();
    } else if (m < p.M) {
      float old[32];
#pragma unroll
      for (int j = 0; j < 32; ++j)
        old[j] = (p.beta != 0.f && nb + j < p.N) ? crow[(long long)(nb + j) * p.cn] : 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = nb + j;
        if (n < p.N) {
          const float v = nk > 0 ? __uint_as_float(r[j]) : 0.f;  // an empty K range adds nothing
          crow[(long long)n * p.cn] = p.beta != 0.f ? fmaf(p.beta, old[j], v) : v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
  }
}

// FP32 product with general strides (the network's full-precision mode):
// C[bz](m, n) = sum_k A(m, k) B(k, n) (+ beta C), A(m, k) at
// a + b * sa + m * am + k * ak, B(k, n) at bb + b * sb + k * bk + n * bn.
// 64 x 64 tiles, 256 threads, 4 x 4 outputs per thread, 16-deep K slabs.
__global__ void __launch_bounds__(256)
gemm_f32_kernel(const float *__restrict__ a, long long am, long long ak, long long sa, const float *__restrict__ bb,
                long long bk, long long bn, long long sb, float *__restrict__ c, long long cm, long long cn,
                long long sc, int M, int N, int K, float beta) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64, b = blockIdx.z;
  a += (long long)b * sa;
  bb += (long long)b * sb;
  c += (long long)b * sc;
  float acc[4][4] = {};
  for (int kk = 0; kk < K; kk += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kq = e / 64, r = e % 64;
      const int m = m0 + r, n = n0 + r, k = kk + kq;
      As[kq][r] = (m < M && k < K) ? a[(long long)m * am + (long long)k * ak] : 0.f;
      Bs[kq][r] = (n < N && k < K) ? bb[(long long)k * bk + (long long)n * bn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kq = 0; kq < 16; ++kq) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = As[kq][ty + 16 * i];
        bv[i] = Bs[kq][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        float *d = c + (long long)m * cm + (long long)n * cn;
        *d = beta != 0.f ? fmaf(beta, *d, acc[i][j]) : acc[i][j];
      }
    }
}

typedef CUresult (*encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 3D map {K, rows, batch} of a BF16 operand, box {64, box_rows, 1},
// 128-byte swizzle, zero fill outside.
cudaError_t operand_map(const __nv_bfloat16 *base, int K, int rows, int ld, long long sb, int nb, int box_rows,
                        CUtensorMap *map) {
  static encode_tiled_fn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (encode_tiled_fn)fn;
  }
  const long long row_bytes = (long long)ld * 2;
  long long batch_bytes = sb * 2;
  if (nb <= 1) batch_bytes = ((row_bytes * rows + 15) / 16) * 16;  // unused dimension
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)std::max(nb, 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)batch_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(base), dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int kStages>
cudaError_t launch_tn(const CUtensorMap &mx, const CUtensorMap &my, const GemmParams &p, int nb, cudaStream_t st) {
  const size_t smem = sizeof(Smem<BN, kStages>) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tn_bf16_kernel<BN, kStages>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((p.M + kBM - 1) / kBM), (unsigned)((p.N + BN - 1) / BN), (unsigned)(nb * p.ksplit));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, gemm_tn_bf16_kernel<BN, kStages>, mx, my, p);
}

template <int BN>
cudaError_t launch_tn_stages(const CUtensorMap &mx, const CUtensorMap &my, const GemmParams &p, int nb,
                             cudaStream_t st) {
  return p.kper <= kBK ? launch_tn<BN, 1>(mx, my, p, nb, st) : launch_tn<BN, 4>(mx, my, p, nb, st);
}

}  // namespace

cudaError_t gemm_tn_bf16(const __nv_bfloat16 *X, int ldx, long long sX, const __nv_bfloat16 *Y, int ldy, long long sY,
                         float *C, long long cm, long long cn, long long sC, int M, int N, int K, int batch, int ksplit,
                         float beta, int *err, cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1 || batch < 1 || ksplit < 1) return cudaErrorInvalidValue;
  if ((ldx % 8) || (ldy % 8) || (sX % 8) || (sY % 8) || ldx < K || ldy < K) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Y) & 15)) return cudaErrorInvalidValue;
  const int BN = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  CUtensorMap mx, my;
  cudaError_t e = operand_map(X, K, M, ldx, sX, sX ? batch : 1, kBM, &mx);
  if (e == cudaSuccess) e = operand_map(Y, K, N, ldy, sY, sY ? batch : 1, BN, &my);
  if (e != cudaSuccess) return e;
  GemmParams p{};
  p.M = M;
  p.N = N;
  p.K = K;
  p.ksplit = ksplit;
  p.kper = ((K + ksplit - 1) / ksplit + kBK - 1) / kBK * kBK;
  p.x_batched = sX != 0;
  p.y_batched = sY != 0;
  p.c = C;
  p.cm = cm;
  p.cn = cn;
  p.sC = sC;
  p.beta = beta;
  p.err = err;
  switch (BN) {
    case 32: return launch_tn_stages<32>(mx, my, p, batch, st);
    case 64: return launch_tn_stages<64>(mx, my, p, batch, st);
    case 128: return launch_tn_stages<128>(mx, my, p, batch, st);
    default: return launch_tn_stages<256>(mx, my, p, batch, st);
  }
}

cudaError_t gemm_f32(const float *A, long long am, long long ak, long long sA, const float *B, long long bk,
                     long long bn, long long sB, float *C, long long cm, long long cn, long long sC, int M, int N,
                     int K, int batch, float beta, cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1 || batch < 1) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)batch);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, gemm_f32_kernel, A, am, ak, sA, B, bk, bn, sB, C, cm, cn, sC, M, N, K, beta);
}

}  // namespace tc

extern "C" int fno_gemm_bf16(const void *X, int32_t ldx, int64_t sX, const void *Y, int32_t ldy, int64_t sY, float *C,
                             int64_t cm, int64_t cn, int64_t sC, int32_t M, int32_t N, int32_t K, int32_t batch,
                             float beta, int *err, void *stream) {
  if (!X || !Y || !C || !err) return LB_ERR_ARG;
  const cudaError_t e = tc::gemm_tn_bf16((const __nv_bfloat16 *)X, ldx, sX, (const __nv_bfloat16 *)Y, ldy, sY, C, cm,
                                         cn, sC, M, N, K, batch, 1, beta, err, (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return LB_ERR_ARG;
  return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
