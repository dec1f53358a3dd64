// gemm_tc.h -- matrix products of the network (see gemm_tc.cu).  Internal
// to the library; not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace tc {

struct GemmParams {
  int M, N, K;
  int ksplit, kper;           // K split into ksplit ranges of kper (multiple of 64)
  int x_batched, y_batched;   // operand has a batch dimension (else shared by all batches)
  float *c;                   // output: element (bz, m, n) at c + bz * sC + m * cm + n * cn
  long long cm, cn, sC;
  float beta;                 // C = D + beta * C
  int *err;                   // set to 1 when a bounded wait gives up
};

// D[b](m, n) = sum_k X[b](m, k) Y[b](n, k) on the tensor cores: X is M x K
// with row pitch ldx (elements) and batch stride sX (0: one matrix for all
// batches), Y is N x K with ldy, sY; both BF16 with k contiguous, pitches and
// strides multiples of 8 elements and 16-byte aligned bases.  FP32 result
// C = D + beta * C; with ksplit > 1 the K range is split and batch-split
// index b * ksplit + s writes its partial product to slice b * ksplit + s.
cudaError_t gemm_tn_bf16(const __nv_bfloat16 *X, int ldx, long long sX, const __nv_bfloat16 *Y, int ldy, long long sY,
                         float *C, long long cm, long long cn, long long sC, int M, int N, int K, int batch, int ksplit,
                         float beta, int *err, cudaStream_t st);

// FP32 product with general strides: C[b](m, n) = sum_k A(m, k) B(k, n)
// (+ beta C), A(m, k) at A + b sA + m am + k ak, B(k, n) at B + b sB + k bk
// + n bn, C(m, n) at C + b sC + m cm + n cn.
cudaError_t gemm_f32(const float *A, long long am, long long ak, long long sA, const float *B, long long bk,
                     long long bn, long long sB, float *C, long long cm, long long cn, long long sC, int M, int N,
                     int K, int batch, float beta, cudaStream_t st);

}  // namespace tc
