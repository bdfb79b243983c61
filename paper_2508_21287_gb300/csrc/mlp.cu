// Cardinality model: a 3-layer MLP (32 -> 128 -> 128 -> 1, ReLU) that predicts the log growth
// of the intermediate table for a candidate join step, trained on the cardinalities the
// executor logs. Matmuls run on the tensor cores as BF16 x BF16 -> FP32 (mma.m16n8k16); the
// master weights, biases, the output layer and Adam's moments stay FP32. Activations that
// feed a matmul are rounded to BF16 (round to nearest even) right after they are produced.
//
// Flat parameter layout (FP32): W1[128][32] | b1[128] | W2[128][128] | b2[128] | w3[128] | b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace dmk {

constexpr int MLP_IN = 32, MLP_H = 128;

// C[M x N] (+)= sum_k A(m, k) * B(k, n); A(m, k) = A[m * am + k * ak], B(k, n) = B[k * bk + n * bn],
// M % 16 == 0, N % 8 == 0, K % 16 == 0. One warp per 16 x 8 tile of C.
__global__ void k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, int am, int ak, const __nv_bfloat16 *Bm,
                            int bk, int bn, float *C, int ldc, int accumulate) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = N / 8;
  if (warp >= (M / 16) * tiles_n) return;
  const int m0 = (warp / tiles_n) * 16, n0 = (warp % tiles_n) * 8;
  const int g = lane >> 2, t = lane & 3;
  float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
  auto ld = [](const __nv_bfloat16 *p, int64_t i) { return __bfloat16_as_ushort(p[i]); };
  for (int k0 = 0; k0 < K; k0 += 16) {
    auto a_at = [&](int r, int c) { return ld(A, (int64_t)(m0 + r) * am + (int64_t)(k0 + c) * ak); };
    auto b_at = [&](int r, int c) { return ld(Bm, (int64_t)(k0 + r) * bk + (int64_t)(n0 + c) * bn); };
    uint32_t a0 = a_at(g, 2 * t) | ((uint32_t)a_at(g, 2 * t + 1) << 16);
    uint32_t a1 = a_at(g + 8, 2 * t) | ((uint32_t)a_at(g + 8, 2 * t + 1) << 16);
    uint32_t a2 = a_at(g, 2 * t + 8) | ((uint32_t)a_at(g, 2 * t + 9) << 16);
    uint32_t a3 = a_at(g + 8, 2 * t + 8) | ((uint32_t)a_at(g + 8, 2 * t + 9) << 16);
    uint32_t b0 = b_at(2 * t, g) | ((uint32_t)b_at(2 * t + 1, g) << 16);
    uint32_t b1 = b_at(2 * t + 8, g) | ((uint32_t)b_at(2 * t + 9, g) << 16);
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float *c0 = C + (int64_t)(m0 + g) * ldc + n0 + 2 * t;
  float *c1 = C + (int64_t)(m0 + g + 8) * ldc + n0 + 2 * t;
  if (accumulate) {
    c0[0] += d0;
    c0[1] += d1;
    c1[0] += d2;
    c1[1] += d3;
  } else {
    c0[0] = d0;
    c0[1] = d1;
    c1[0] = d2;
    c1[1] = d3;
  }
}

__global__ void k_to_bf16(const float *x, __nv_bfloat16 *y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// H = relu(Z + b) rounded to BF16; Z keeps the pre-activation (its sign is the ReLU mask).
__global__ void k_bias_relu(float *Z, const float *b, __nv_bfloat16 *H, int rows, int cols) {
  int64_t n = (int64_t)rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float z = Z[i] + b[i % cols];
    Z[i] = z;
    H[i] = __float2bfloat16_rn(z > 0.f ? z : 0.f);
  }
}

// y[r] = sum_o H2[r][o] * w3[o] + b3 (FP32); with targets, dy[r] = 2 (y - t) / n_valid for valid rows
// and the squared error is added to *loss.
__global__ void k_out_layer(const __nv_bfloat16 *H2, const float *w3, const float *b3, int rows, int n_valid,
                            const float *target, float *y, float *dy, float *loss) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (r >= rows) return;
  float s = 0.f;
  for (int o = lane; o < MLP_H; o += 32) s += __bfloat162float(H2[(int64_t)r * MLP_H + o]) * w3[o];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) {
    float v = s + b3[0];
    y[r] = v;
    if (target) {
      float e = r < n_valid ? v - target[r] : 0.f;
      dy[r] = 2.f * e / (float)n_valid;
      if (r < n_valid) atomicAdd(loss, e * e / (float)n_valid);
    }
  }
}

// dH2 = dy * w3 masked by Z2 > 0 (BF16); also dw3 and db3 (FP32, accumulated).
__global__ void k_out_backward(const float *dy, const __nv_bfloat16 *H2, const float *Z2, const float *w3, int rows,
                               __nv_bfloat16 *dH2, float *dw3, float *db3) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < MLP_H) {
    float s = 0.f;
    for (int r = 0; r < rows; r++) s += dy[r] * __bfloat162float(H2[(int64_t)r * MLP_H + o]);
    dw3[o] += s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int r = 0; r < rows; r++) s += dy[r];
    db3[0] += s;
  }
  int64_t n = (int64_t)rows * MLP_H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / MLP_H;
    int oo = (int)(i - r * MLP_H);
    float g = Z2[i] > 0.f ? dy[r] * w3[oo] : 0.f;
    dH2[i] = __float2bfloat16_rn(g);
  }
}

// dH = dA masked by Z > 0, rounded to BF16.
__global__ void k_relu_backward(const float *dA, const float *Z, __nv_bfloat16 *dH, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dH[i] = __float2bfloat16_rn(Z[i] > 0.f ? dA[i] : 0.f);
}

// db[c] += sum_r dH[r][c]
__global__ void k_colsum(const __nv_bfloat16 *dH, int rows, int cols, float *db) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; r++) s += __bfloat162float(dH[(int64_t)r * cols + c]);
  db[c] += s;
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

static int blocks_for(int64_t n, int per = 256) {
  int64_t b = (n + per - 1) / per;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

static cudaError_t gemm(int M, int N, int K, const __nv_bfloat16 *A, int am, int ak, const __nv_bfloat16 *Bm, int bk,
                        int bn, float *C, int ldc, int acc, cudaStream_t s) {
  int warps = (M / 16) * (N / 8);
  int threads = 128;
  int blocks = (warps * 32 + threads - 1) / threads;
  g_launches++;
  k_gemm_bf16<<<blocks, threads, 0, s>>>(M, N, K, A, am, ak, Bm, bk, bn, C, ldc, acc);
  return cudaGetLastError();
}

int64_t mlp_param_count() { return (int64_t)MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1; }

int64_t mlp_work_bytes(int rows) {
  int64_t r = rows;
  return r * MLP_IN * 2 + 2 * (r * MLP_H * 4) + 2 * (r * MLP_H * 2) + 3 * r * 4 + 2 * (r * MLP_H * 2) +
         r * MLP_H * 4 + 2 * mlp_param_count() * 2 + 4096;
}

// Forward (and, with targets, backward into grads) for `rows` samples (rows % 16 == 0; the
// first n_valid are real). X: rows x 32 FP32 on the device; params / grads: flat FP32.
cudaError_t mlp_forward_backward(const float *params, const float *X, const float *target, int rows, int n_valid,
                                 float *y, float *grads, float *loss, void *work, cudaStream_t s) {
  const float *W1 = params, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
  const float *w3 = b2 + MLP_H, *b3 = w3 + MLP_H;
  unsigned char *p = (unsigned char *)work;
  auto take = [&](int64_t bytes) {
    void *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  __nv_bfloat16 *Xb = (__nv_bfloat16 *)take((int64_t)rows * MLP_IN * 2);
  float *Z1 = (float *)take((int64_t)rows * MLP_H * 4);
  float *Z2 = (float *)take((int64_t)rows * MLP_H * 4);
  __nv_bfloat16 *H1 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  __nv_bfloat16 *H2 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  float *dy = (float *)take((int64_t)rows * 4);
  __nv_bfloat16 *dH2 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  __nv_bfloat16 *dH1 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  float *dA1 = (float *)take((int64_t)rows * MLP_H * 4);
  __nv_bfloat16 *W1b = (__nv_bfloat16 *)take((int64_t)MLP_H * MLP_IN * 2);
  __nv_bfloat16 *W2b = (__nv_bfloat16 *)take((int64_t)MLP_H * MLP_H * 2);
  int launches = 0;
  k_to_bf16<<<blocks_for((int64_t)rows * MLP_IN), 256, 0, s>>>(X, Xb, (int64_t)rows * MLP_IN);
  k_to_bf16<<<blocks_for(MLP_H * MLP_IN), 256, 0, s>>>(W1, W1b, MLP_H * MLP_IN);
  k_to_bf16<<<blocks_for(MLP_H * MLP_H), 256, 0, s>>>(W2, W2b, MLP_H * MLP_H);
  launches += 3;
  // Z1 = X W1^T: A = X (row-major), B(k, n) = W1[n][k]
  cudaError_t e = gemm(rows, MLP_H, MLP_IN, Xb, MLP_IN, 1, W1b, 1, MLP_IN, Z1, MLP_H, 0, s);
  if (e != cudaSuccess) return e;
  k_bias_relu<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(Z1, b1, H1, rows, MLP_H);
  e = gemm(rows, MLP_H, MLP_H, H1, MLP_H, 1, W2b, 1, MLP_H, Z2, MLP_H, 0, s);
  if (e != cudaSuccess) return e;
  k_bias_relu<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(Z2, b2, H2, rows, MLP_H);
  k_out_layer<<<(rows + 7) / 8, 256, 0, s>>>(H2, w3, b3, rows, n_valid, target, y, dy, loss);
  launches += 3;
  if (target && grads) {
    float *gW1 = grads, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    float *gw3 = gb2 + MLP_H, *gb3 = gw3 + MLP_H;
    k_out_backward<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(dy, H2, Z2, w3, rows, dH2, gw3, gb3);
    k_colsum<<<1, MLP_H, 0, s>>>(dH2, rows, MLP_H, gb2);
    launches += 2;
    // gW2[o][i] += sum_r dH2[r][o] H1[r][i]: A(m=o, k=r) = dH2[r][o], B(k=r, n=i) = H1[r][i]
    e = gemm(MLP_H, MLP_H, rows, dH2, 1, MLP_H, H1, MLP_H, 1, gW2, MLP_H, 1, s);
    if (e != cudaSuccess) return e;
    // dA1[r][i] = sum_o dH2[r][o] W2[o][i]: A = dH2 (row-major), B(k=o, n=i) = W2[o][i]
    e = gemm(rows, MLP_H, MLP_H, dH2, MLP_H, 1, W2b, MLP_H, 1, dA1, MLP_H, 0, s);
    if (e != cudaSuccess) return e;
    k_relu_backward<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(dA1, Z1, dH1, (int64_t)rows * MLP_H);
    k_colsum<<<1, MLP_H, 0, s>>>(dH1, rows, MLP_H, gb1);
    launches += 2;
    // gW1[o][j] += sum_r dH1[r][o] X[r][j]
    e = gemm(MLP_H, MLP_IN, rows, dH1, 1, MLP_H, Xb, MLP_IN, 1, gW1, MLP_IN, 1, s);
    if (e != cudaSuccess) return e;
  }
  g_launches += launches;
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, const float *grads, float *m, float *v, int64_t n, float lr, int step,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  g_launches++;
  k_adam<<<blocks_for(n), 256, 0, s>>>(params, grads, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

}  // namespace dmk
