// Atom-pair MLP for the learned initial density: three dense layers
// (nin -> H -> H -> nout) with SiLU activations, BF16 weights, FP32
// activations and FP32 accumulation; forward, masked mean-squared-error loss
// with backward pass, and an Adam step on FP32 master weights.  Written for
// the SCF extension (no counterpart in the paper).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "fock_impl.h"

struct fock_mlp {
  int nin, H, nout, max_batch;
  size_t nparam;
  // parameters (FP32 master), BF16 copies of the three weight matrices
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *w16 = nullptr;
  // activations for max_batch rows
  float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr, *dy = nullptr;
  float *d1 = nullptr, *d2 = nullptr, *loss = nullptr;
  long long step = 0;
  size_t off_w1, off_b1, off_w2, off_b2, off_w3, off_b3;
  size_t o16_w1, o16_w2, o16_w3;
};

namespace {

template <class T>
__device__ __forceinline__ float ld(const T *p) {
  return (float)(*p);
}
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}

// Round an FP32 value to TF32 (10-bit mantissa, round to nearest away) and
// return it as its 32-bit pattern, the operand format of mma .tf32.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// D = A B + C for one m16n8k8 tile on the tensor cores (TF32 inputs, FP32
// accumulation; fragment layouts of the PTX ISA for mma.m16n8k8 .tf32).
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[m][n] (+)= sum_k A(m,k) B(k,n); A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n], on the tensor cores: a block of four
// warps owns a 64 x 64 tile of C (each warp 32 x 32, 2 x 4 mma tiles), K in
// steps of 16 staged in shared memory as FP32.  Each operand is split into a
// TF32 high part and a TF32 remainder, and the three products hi*hi, hi*lo,
// lo*hi are accumulated in FP32, which keeps the product accurate to about
// FP32 rounding (BF16 weights are exact in TF32, so their remainder is zero).
// Optional epilogue: + bias[n], store pre- and post-SiLU values.
constexpr int GT = 64, GK = 16;
template <bool TA, bool TB, class TAt, class TBt>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const TAt *__restrict__ A, int lda,
                                              const TBt *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                              int accumulate, const float *__restrict__ bias, float *__restrict__ act) {
  __shared__ float As[GT][GK + 4];  // [m][k]
  __shared__ float Bs[GT][GK + 4];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int i = tid; i < GT * GK; i += 128) {
      const int r = i / GK, k = i - r * GK;  // k fastest: row-major reads of A and B^T
      const int m = m0 + r, n = n0 + r, kk = k0 + k;
      As[r][k] = (m < M && kk < K) ? ld(TA ? A + (size_t)kk * lda + m : A + (size_t)m * lda + kk) : 0.0f;
      Bs[r][k] = (n < N && kk < K) ? ld(TB ? B + (size_t)n * ldb + kk : B + (size_t)kk * ldb + n) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GK; ks += 8) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        const float v[4] = {As[r][ks + t], As[r + 8][ks + t], As[r][ks + t + 4], As[r + 8][ks + t + 4]};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ah[i][q] = to_tf32(v[q]);
          al[i][q] = to_tf32(v[q] - __uint_as_float(ah[i][q]));
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + g;
        const float v[2] = {Bs[c][ks + t], Bs[c][ks + t + 4]};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          bh[j][q] = to_tf32(v[q]);
          bl[j][q] = to_tf32(v[q] - __uint_as_float(bh[j][q]));
        }
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          mma_tf32(acc[i][j], al[i], bh[j]);
          mma_tf32(acc[i][j], ah[i], bl[j]);
          mma_tf32(acc[i][j], ah[i], bh[j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0), col = n0 + wn + 8 * j + 2 * t + (r & 1);
        if (row >= M || col >= N) continue;
        float v = acc[i][j][r];
        if (bias) v += bias[col];
        float *c = C + (size_t)row * ldc + col;
        *c = accumulate ? *c + v : v;
        if (act) {
          const float s = 1.0f / (1.0f + __expf(-v));
          act[(size_t)row * ldc + col] = v * s;
        }
      }
}

// d = dA * silu'(z)
__global__ void k_silu_bwd(long long n, const float *__restrict__ z, const float *__restrict__ da,
                           float *__restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float s = 1.0f / (1.0f + __expf(-z[i]));
    d[i] = da[i] * s * (1.0f + z[i] * (1.0f - s));
  }
}

// db[n] += sum_b d[b][n]
__global__ void k_colsum(int B, int N, const float *__restrict__ d, float *__restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.0f;
  for (int b = 0; b < B; ++b) s += d[(size_t)b * N + n];
  db[n] += s;
}

// masked MSE: loss += sum mask (y - t)^2 / norm, dy = 2 mask (y - t) / norm
__global__ void k_loss(long long n, const float *__restrict__ y, const float *__restrict__ t,
                       const float *__restrict__ mask, float inv_norm, float *__restrict__ dy, float *__restrict__ loss) {
  float s = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float w = mask ? mask[i] : 1.0f;
    const float r = (y[i] - t[i]) * w;
    dy[i] = 2.0f * r * inv_norm;
    s += r * (y[i] - t[i]) * inv_norm;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

__global__ void k_adam(long long n, float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float wd, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] + wd * p[i];
    m[i] = b1 * m[i] + (1.0f - b1) * gi;
    v[i] = b2 * v[i] + (1.0f - b2) * gi * gi;
    p[i] -= lr * (m[i] * c1) / (sqrtf(v[i] * c2) + eps);
    g[i] = 0.0f;
  }
}

__global__ void k_to_bf16(long long n, const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

template <bool TA, bool TB, class TAt, class TBt>
cudaError_t gemm(int M, int N, int K, const TAt *A, int lda, const TBt *B, int ldb, float *C, int ldc, int acc,
                 const float *bias, float *act, cudaStream_t st) {
  dim3 grd((N + GT - 1) / GT, (M + GT - 1) / GT);
  k_gemm<TA, TB, TAt, TBt><<<grd, 128, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, acc, bias, act);
  return cudaGetLastError();
}

cudaError_t refresh_bf16(fock_mlp *n, cudaStream_t st) {
  k_to_bf16<<<blocks_for((long long)n->H * n->nin), 256, 0, st>>>((long long)n->H * n->nin, n->p + n->off_w1,
                                                                   n->w16 + n->o16_w1);
  k_to_bf16<<<blocks_for((long long)n->H * n->H), 256, 0, st>>>((long long)n->H * n->H, n->p + n->off_w2,
                                                                 n->w16 + n->o16_w2);
  k_to_bf16<<<blocks_for((long long)n->nout * n->H), 256, 0, st>>>((long long)n->nout * n->H, n->p + n->off_w3,
                                                                   n->w16 + n->o16_w3);
  return cudaGetLastError();
}

cudaError_t forward(fock_mlp *n, const float *X, int B, float *Y, cudaStream_t st) {
  const int H = n->H;
  cudaError_t e = gemm<false, true>(B, H, n->nin, X, n->nin, n->w16 + n->o16_w1, n->nin, n->z1, H, 0, n->p + n->off_b1,
                                    n->a1, st);
  if (e == cudaSuccess)
    e = gemm<false, true>(B, H, H, (const float *)n->a1, H, n->w16 + n->o16_w2, H, n->z2, H, 0, n->p + n->off_b2, n->a2,
                          st);
  if (e == cudaSuccess)
    e = gemm<false, true>(B, n->nout, H, (const float *)n->a2, H, n->w16 + n->o16_w3, H, Y, n->nout, 0,
                          n->p + n->off_b3, (float *)nullptr, st);
  return e;
}

fock_status st_of(cudaError_t e) {
  if (e == cudaSuccess) return FOCK_OK;
  return e == cudaErrorMemoryAllocation ? FOCK_ERR_OOM : FOCK_ERR_CUDA;
}

}  // namespace

extern "C" {

fock_status fock_mlp_create(int32_t nin, int32_t nhidden, int32_t nout, int32_t max_batch, uint64_t seed,
                            fock_mlp **out) {
  if (!out || nin < 1 || nhidden < 1 || nout < 1 || max_batch < 1) return FOCK_ERR_INVALID_ARG;
  *out = nullptr;
  fock_mlp *n = new (std::nothrow) fock_mlp();
  if (!n) return FOCK_ERR_OOM;
  n->nin = nin;
  n->H = nhidden;
  n->nout = nout;
  n->max_batch = max_batch;
  const size_t H = nhidden;
  n->off_w1 = 0;
  n->off_b1 = n->off_w1 + H * nin;
  n->off_w2 = n->off_b1 + H;
  n->off_b2 = n->off_w2 + H * H;
  n->off_w3 = n->off_b2 + H;
  n->off_b3 = n->off_w3 + (size_t)nout * H;
  n->nparam = n->off_b3 + nout;
  n->o16_w1 = 0;
  n->o16_w2 = H * nin;
  n->o16_w3 = n->o16_w2 + H * H;
  const size_t n16 = n->o16_w3 + (size_t)nout * H;
  const size_t act = (size_t)max_batch * (4 * H + 2 * (size_t)nout + 2 * H);
  float *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(float) * (4 * n->nparam + act + 1) + sizeof(__nv_bfloat16) * n16);
  if (e != cudaSuccess) {
    delete n;
    return st_of(e);
  }
  n->p = buf;
  n->g = n->p + n->nparam;
  n->m = n->g + n->nparam;
  n->v = n->m + n->nparam;
  float *a = n->v + n->nparam;
  const size_t B = max_batch;
  n->z1 = a;
  n->a1 = n->z1 + B * H;
  n->z2 = n->a1 + B * H;
  n->a2 = n->z2 + B * H;
  n->y = n->a2 + B * H;
  n->dy = n->y + B * nout;
  n->d1 = n->dy + B * nout;
  n->d2 = n->d1 + B * H;
  n->loss = n->d2 + B * H;
  n->w16 = (__nv_bfloat16 *)(n->loss + 1);
  // He-style initialisation from a 64-bit LCG (host), biases zero
  std::vector<float> p(n->nparam, 0.0f);
  uint64_t s = seed * 6364136223846793005ull + 1442695040888963407ull;
  auto uni = [&]() {
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(s >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](size_t off, size_t cnt, int fan_in) {
    const double r = sqrt(3.0 / fan_in);
    for (size_t i = 0; i < cnt; ++i) p[off + i] = (float)((2.0 * uni() - 1.0) * r);
  };
  fill(n->off_w1, H * nin, nin);
  fill(n->off_w2, H * H, (int)H);
  fill(n->off_w3, (size_t)nout * H, (int)H);
  e = cudaMemcpy(n->p, p.data(), sizeof(float) * n->nparam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->g, 0, sizeof(float) * 3 * n->nparam);
  if (e == cudaSuccess) e = refresh_bf16(n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(buf);
    delete n;
    return st_of(e);
  }
  *out = n;
  return FOCK_OK;
}

fock_status fock_mlp_free(fock_mlp *n) {
  if (!n) return FOCK_OK;
  cudaFree(n->p);
  delete n;
  return FOCK_OK;
}

int64_t fock_mlp_num_params(const fock_mlp *n) { return n ? (int64_t)n->nparam : -1; }

fock_status fock_mlp_get_params(const fock_mlp *n, float *host_params, float *host_grads) {
  if (!n) return FOCK_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (host_params) e = cudaMemcpy(host_params, n->p, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && host_grads) e = cudaMemcpy(host_grads, n->g, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost);
  return st_of(e);
}

fock_status fock_mlp_set_params(fock_mlp *n, const float *host_params) {
  if (!n || !host_params) return FOCK_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpy(n->p, host_params, sizeof(float) * n->nparam, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = refresh_bf16(n, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return st_of(e);
}

fock_status fock_mlp_forward(fock_mlp *n, const float *X, int32_t B, float *Y, cudaStream_t st) {
  if (!n || !X || !Y || B < 0 || B > n->max_batch) return FOCK_ERR_INVALID_ARG;
  if (B == 0) return FOCK_OK;
  return st_of(forward(n, X, B, Y, st));
}

fock_status fock_mlp_loss_backward(fock_mlp *n, const float *X, const float *T, const float *mask, int32_t B,
                                   double norm, float *loss_host, cudaStream_t st) {
  if (!n || !X || !T || B < 1 || B > n->max_batch || !(norm > 0.0)) return FOCK_ERR_INVALID_ARG;
  const int H = n->H, O = n->nout;
  cudaError_t e = cudaMemsetAsync(n->loss, 0, sizeof(float), st);
  if (e == cudaSuccess) e = forward(n, X, B, n->y, st);
  const long long ny = (long long)B * O;
  if (e == cudaSuccess) {
    k_loss<<<blocks_for(ny), 256, 0, st>>>(ny, n->y, T, mask, (float)(1.0 / norm), n->dy, n->loss);
    e = cudaGetLastError();
  }
  // layer 3: dW3 += dy^T a2, db3 += colsum(dy), da2 = dy W3
  if (e == cudaSuccess)
    e = gemm<true, false>(O, H, B, (const float *)n->dy, O, (const float *)n->a2, H, n->g + n->off_w3, H, 1,
                          (const float *)nullptr, (float *)nullptr, st);
  if (e == cudaSuccess) {
    k_colsum<<<(O + 127) / 128, 128, 0, st>>>(B, O, n->dy, n->g + n->off_b3);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = gemm<false, false>(B, H, O, (const float *)n->dy, O, n->w16 + n->o16_w3, H, n->d2, H, 0,
                           (const float *)nullptr, (float *)nullptr, st);
  const long long nh = (long long)B * H;
  if (e == cudaSuccess) {
    k_silu_bwd<<<blocks_for(nh), 256, 0, st>>>(nh, n->z2, n->d2, n->d2);
    e = cudaGetLastError();
  }
  // layer 2
  if (e == cudaSuccess)
    e = gemm<true, false>(H, H, B, (const float *)n->d2, H, (const float *)n->a1, H, n->g + n->off_w2, H, 1,
                          (const float *)nullptr, (float *)nullptr, st);
  if (e == cudaSuccess) {
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(B, H, n->d2, n->g + n->off_b2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = gemm<false, false>(B, H, H, (const float *)n->d2, H, n->w16 + n->o16_w2, H, n->d1, H, 0,
                           (const float *)nullptr, (float *)nullptr, st);
  if (e == cudaSuccess) {
    k_silu_bwd<<<blocks_for(nh), 256, 0, st>>>(nh, n->z1, n->d1, n->d1);
    e = cudaGetLastError();
  }
  // layer 1
  if (e == cudaSuccess)
    e = gemm<true, false>(H, n->nin, B, (const float *)n->d1, H, X, n->nin, n->g + n->off_w1, n->nin, 1,
                          (const float *)nullptr, (float *)nullptr, st);
  if (e == cudaSuccess) {
    k_colsum<<<(H + 127) / 128, 128, 0, st>>>(B, H, n->d1, n->g + n->off_b1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && loss_host) {
    e = cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return st_of(e);
}

fock_status fock_mlp_step(fock_mlp *n, float lr, float beta1, float beta2, float eps, float weight_decay,
                          cudaStream_t st) {
  if (!n || !(lr >= 0.0f)) return FOCK_ERR_INVALID_ARG;
  n->step += 1;
  const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)n->step)));
  const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)n->step)));
  k_adam<<<blocks_for((long long)n->nparam), 256, 0, st>>>((long long)n->nparam, n->p, n->g, n->m, n->v, lr, beta1,
                                                           beta2, eps, weight_decay, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = refresh_bf16(n, st);
  return st_of(e);
}

fock_status fock_mlp_zero_grad(fock_mlp *n, cudaStream_t st) {
  if (!n) return FOCK_ERR_INVALID_ARG;
  return st_of(cudaMemsetAsync(n->g, 0, sizeof(float) * n->nparam, st));
}

}  // extern "C"
