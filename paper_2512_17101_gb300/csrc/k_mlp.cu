// Learned initial guess for the mixture temperature solve (no counterpart in the
// paper; a requirement of the learned form): an 8 -> 64 -> 64 -> 1 tanh MLP that
// maps (normalised e, Y_1..Y_7) to a normalised temperature.
//
//   * training, FP32: per-sample forward and backward passes, gradients summed
//     over each block's samples in shared memory and added to the batch gradient,
//     then an Adam update; samples come from the Newton solver;
//   * inference, FP16 operands with FP32 accumulation on the tensor cores
//     (mma.sync m16n8k16), fused with the FP64 Newton iteration that it seeds:
//     Newton stays the arbiter and the fallback, to the same |dT| < tol.
//
// Flat parameter layout (float): W1 [64][8] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64] | b3.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_newton.cuh"

namespace dg {
namespace {

constexpr int NI = 8, NH = 64;
constexpr int P_W1 = 0, P_B1 = 512, P_W2 = 576, P_B2 = 4672, P_W3 = 4736, P_B3 = 4800;
static_assert(P_B3 + 1 == DG_MLP_PARAMS, "parameter layout");

// ---- training ----------------------------------------------------------------------------------
constexpr int TS = 128;  // samples per block
constexpr int HS = 65;   // padded row of the per-sample activation tables

__global__ void __launch_bounds__(TS) mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ X,
                                                      const float* __restrict__ tgt, int64_t n, float inv_batch,
                                                      float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* sW = sm;                    // DG_MLP_PARAMS
  float* sX = sW + DG_MLP_PARAMS;    // TS x 8
  float* sH1 = sX + TS * NI;         // TS x HS
  float* sH2 = sH1 + TS * HS;
  float* sD1 = sH2 + TS * HS;
  float* sD2 = sD1 + TS * HS;
  float* sdy = sD2 + TS * HS;        // TS
  float* sred = sdy + TS;            // 32
  const int s = threadIdx.x;
  for (int i = s; i < DG_MLP_PARAMS; i += blockDim.x) sW[i] = theta[i];
  const int64_t idx = (int64_t)blockIdx.x * TS + s;
  const bool valid = idx < n;
#pragma unroll
  for (int k = 0; k < NI; ++k) sX[s * NI + k] = valid ? X[idx * NI + k] : 0.0f;
  __syncthreads();
  const float* W1 = sW + P_W1;
  const float* b1 = sW + P_B1;
  const float* W2 = sW + P_W2;
  const float* b2 = sW + P_B2;
  const float* W3 = sW + P_W3;
  float x[NI];
#pragma unroll
  for (int k = 0; k < NI; ++k) x[k] = sX[s * NI + k];
  float h1[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float a = b1[j];
#pragma unroll
    for (int k = 0; k < NI; ++k) a = fmaf(W1[j * NI + k], x[k], a);
    h1[j] = tanhf(a);
    sH1[s * HS + j] = h1[j];
  }
  float y = sW[P_B3];
  for (int i = 0; i < NH; ++i) {
    float a = b2[i];
#pragma unroll
    for (int j = 0; j < NH; ++j) a = fmaf(W2[i * NH + j], h1[j], a);
    const float h = tanhf(a);
    sH2[s * HS + i] = h;
    y = fmaf(W3[i], h, y);
  }
  const float r = valid ? y - tgt[idx] : 0.0f;
  const float dy = 2.0f * r * inv_batch;
  sdy[s] = dy;
  float d1[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) d1[j] = 0.0f;
  for (int i = 0; i < NH; ++i) {
    const float h = sH2[s * HS + i];
    const float d2 = dy * W3[i] * (1.0f - h * h);
    sD2[s * HS + i] = d2;
#pragma unroll
    for (int j = 0; j < NH; ++j) d1[j] = fmaf(W2[i * NH + j], d2, d1[j]);
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) sD1[s * HS + j] = d1[j] * (1.0f - h1[j] * h1[j]);
  // batch loss
  float l = r * r * inv_batch;
#pragma unroll
  for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((s & 31) == 0) sred[s >> 5] = l;
  __syncthreads();
  if (s == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w];
    atomicAdd(loss, t);
  }
  // gradient sums over the block's samples
  for (int e = s; e < DG_MLP_PARAMS; e += blockDim.x) {
    float acc = 0.0f;
    if (e < P_B1) {
      const int j = e / NI, k = e - j * NI;
      for (int t = 0; t < TS; ++t) acc = fmaf(sD1[t * HS + j], sX[t * NI + k], acc);
    } else if (e < P_W2) {
      const int j = e - P_B1;
      for (int t = 0; t < TS; ++t) acc += sD1[t * HS + j];
    } else if (e < P_B2) {
      const int i = (e - P_W2) / NH, j = (e - P_W2) - i * NH;
      for (int t = 0; t < TS; ++t) acc = fmaf(sD2[t * HS + i], sH1[t * HS + j], acc);
    } else if (e < P_W3) {
      const int i = e - P_B2;
      for (int t = 0; t < TS; ++t) acc += sD2[t * HS + i];
    } else if (e < P_B3) {
      const int i = e - P_W3;
      for (int t = 0; t < TS; ++t) acc = fmaf(sdy[t], sH2[t * HS + i], acc);
    } else {
      for (int t = 0; t < TS; ++t) acc += sdy[t];
    }
    atomicAdd(&grad[e], acc);
  }
}

constexpr size_t kGradSmem = sizeof(float) * (DG_MLP_PARAMS + TS * NI + 4 * TS * HS + TS + 32);

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float bc1, float bc2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < DG_MLP_PARAMS; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    grad[i] = 0.0f;
  }
}

// features x = ((e - e_mean)/e_scale, Y_1..Y_ns, 0...), target (T - T_mean)/T_scale
__global__ void features_kernel(int64_t n, int ns, const double* __restrict__ e, const double* __restrict__ Y,
                                const double* __restrict__ T, dg_mlp_norm nrm, float* __restrict__ X,
                                float* __restrict__ t) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    X[i * NI] = (float)((e[i] - nrm.e_mean) / nrm.e_scale);
    for (int k = 0; k < NI - 1; ++k) X[i * NI + 1 + k] = k < ns ? (float)Y[k * n + i] : 0.0f;
    if (T) t[i] = (float)((T[i] - nrm.T_mean) / nrm.T_scale);
  }
}

// FP16 inference weights: W1 [64][16] (k padded with zeros), W2 [64][64]
__global__ void to_half_kernel(const float* __restrict__ theta, __half* __restrict__ w1h, __half* __restrict__ w2h) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH * 16 + NH * NH; i += gridDim.x * blockDim.x) {
    if (i < NH * 16) {
      const int j = i / 16, k = i - j * 16;
      w1h[i] = __float2half_rn(k < NI ? theta[P_W1 + j * NI + k] : 0.0f);
    } else {
      w2h[i - NH * 16] = __float2half_rn(theta[P_W2 + i - NH * 16]);
    }
  }
}

// ---- inference fused with Newton ----------------------------------------------------------------
__device__ __forceinline__ void mma16816h(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Hardware tanh (tanh.approx.f32, about 11 correct bits): the inference only seeds Newton,
// which stays the arbiter of T; training uses the precise tanhf.
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
}

constexpr int W1S = 12;  // words per row of W1 (16 halves + 8 pad)
constexpr int W2S = 36;  // words per row of W2 (64 halves + 8 pad)
constexpr int XS = 12;   // words per row of the input tile

struct MlpDev {
  const uint32_t* w1h;  // [64][8] words
  const uint32_t* w2h;  // [64][32] words
  const float* theta;   // fp32 master (biases, W3)
  dg_mlp_norm nrm;
};

// Per node: the MLP guess (mode DG_TSEED_MLP) or the given seed, then Newton.
// 4 warps per block; each warp handles groups of 32 nodes (two 16-row tiles).
__global__ void __launch_bounds__(128) temperature_mlp_kernel(const GasParams g, const int64_t n,
                                                              const double* __restrict__ q, double* __restrict__ T,
                                                              int32_t* __restrict__ iters, const MlpDev mlp,
                                                              const int guess_only, unsigned* __restrict__ status,
                                                              const MixturePrims mp) {
  __shared__ uint32_t sW1[NH * W1S];
  __shared__ uint32_t sW2[NH * W2S];
  __shared__ float sb1[NH], sb2[NH], sW3[NH];
  __shared__ uint32_t sX[4][32 * XS];
  __shared__ float sY[4][32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gq = lane >> 2, tq = lane & 3;
  for (int i = tid; i < NH * 8; i += blockDim.x) sW1[(i / 8) * W1S + (i % 8)] = mlp.w1h[i];
  for (int i = tid; i < NH * 32; i += blockDim.x) sW2[(i / 32) * W2S + (i % 32)] = mlp.w2h[i];
  for (int i = tid; i < NH; i += blockDim.x) {
    sb1[i] = mlp.theta[P_B1 + i];
    sb2[i] = mlp.theta[P_B2 + i];
    sW3[i] = mlp.theta[P_W3 + i];
  }
  const float b3 = mlp.theta[P_B3];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * 4 * 32;
  for (int64_t g0 = ((int64_t)blockIdx.x * 4 + warp) * 32; g0 < n; g0 += stride) {
    const int64_t node = g0 + lane;
    const bool valid = node < n;
    double e = 0.0, rho = 1.0, Rmix = 0.0, c[6] = {0, 0, 0, 0, 0, 0};
    float feat[NI] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (valid) {
      rho = q[node];
      const double ir = newton::rcp64(rho);
      const double mx = q[n + node], my = q[2 * n + node], mz = q[3 * n + node];
      e = q[4 * n + node] * ir - 0.5 * ir * ir * (mx * mx + my * my + mz * mz);
      feat[0] = (float)((e - mlp.nrm.e_mean) / mlp.nrm.e_scale);
      double Y[DG_MAX_SPECIES];
#pragma unroll
      for (int k = 0; k < DG_MAX_SPECIES; ++k) {
        Y[k] = k < g.ns ? q[(5 + k) * n + node] * ir : 0.0;
        if (k < NI - 1) feat[1 + k] = (float)Y[k];
      }
      newton::fold(g, Y, c, Rmix);
    }
    uint32_t* xr = sX[warp] + lane * XS;
#pragma unroll
    for (int k = 0; k < NI / 2; ++k) xr[k] = pack_half2(feat[2 * k], feat[2 * k + 1]);
#pragma unroll
    for (int k = NI / 2; k < 8; ++k) xr[k] = 0u;
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const uint32_t* x0 = sX[warp] + (mt * 16 + gq) * XS;
      const uint32_t* x1 = sX[warp] + (mt * 16 + gq + 8) * XS;
      const uint32_t a1[4] = {x0[tq], x1[tq], x0[4 + tq], x1[4 + tq]};
      uint32_t a2[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float cc[4] = {0, 0, 0, 0};
        const uint32_t* w = sW1 + (nt * 8 + gq) * W1S;
        mma16816h(cc, a1, w[tq], w[4 + tq]);
        const int col = nt * 8 + 2 * tq;
        const float h0 = tanh_fast(cc[0] + sb1[col]), h1 = tanh_fast(cc[1] + sb1[col + 1]);
        const float h2 = tanh_fast(cc[2] + sb1[col]), h3 = tanh_fast(cc[3] + sb1[col + 1]);
        // accumulator tile nt becomes half of the A fragment of layer-2 k-tile nt/2
        const int kt = nt >> 1, hi = nt & 1;
        a2[kt][hi ? 2 : 0] = pack_half2(h0, h1);
        a2[kt][hi ? 3 : 1] = pack_half2(h2, h3);
      }
      float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float cc[4] = {0, 0, 0, 0};
        const uint32_t* w = sW2 + (nt * 8 + gq) * W2S;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma16816h(cc, a2[kt], w[kt * 8 + tq], w[kt * 8 + 4 + tq]);
        const int col = nt * 8 + 2 * tq;
        y0 = fmaf(sW3[col], tanh_fast(cc[0] + sb2[col]), fmaf(sW3[col + 1], tanh_fast(cc[1] + sb2[col + 1]), y0));
        y1 = fmaf(sW3[col], tanh_fast(cc[2] + sb2[col]), fmaf(sW3[col + 1], tanh_fast(cc[3] + sb2[col + 1]), y1));
      }
      y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
      y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
      y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
      y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
      if (tq == 0) {
        sY[warp][mt * 16 + gq] = y0 + b3;
        sY[warp][mt * 16 + gq + 8] = y1 + b3;
      }
    }
    __syncwarp();
    double t = mlp.nrm.T_mean + mlp.nrm.T_scale * (double)sY[warp][lane];
    t = fmin(fmax(t, mlp.nrm.T_min), mlp.nrm.T_max);
    __syncwarp();
    if (!valid) continue;
    if (guess_only) {
      T[node] = t;
      continue;
    }
    int it;
    double cv;
    if (!newton::solve(c, e, t, g.newton_max_it, g.newton_tol, it, cv)) atomicOr(status, DG_STATUS_NO_CONVERGENCE);
    T[node] = t;
    if (iters) iters[node] = it;
    if (mp.rec) newton::store_prims(mp, g, q, n, node, rho, Rmix, t, cv);
    if (mp.prim) newton::store_prims64(mp, c, n, node, rho, Rmix, t);
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t ensure_half_weights(dg_gas gas) {
  if (!gas->mlp_w1h) {
    cudaError_t e = cudaMalloc((void**)&gas->mlp_w1h, sizeof(__half) * NH * 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&gas->mlp_w2h, sizeof(__half) * NH * NH);
    if (e != cudaSuccess) return e;
  }
  to_half_kernel<<<16, 256>>>(gas->mlp_theta, (__half*)gas->mlp_w1h, (__half*)gas->mlp_w2h);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

}  // namespace

cudaError_t launch_temperature_mlp(dg_gas gas, int64_t n, const double* q, double* T, int32_t* iters, int guess_only,
                                   cudaStream_t s, const MixturePrims& mp) {
  if (n <= 0) return cudaSuccess;
  MlpDev m{(const uint32_t*)gas->mlp_w1h, (const uint32_t*)gas->mlp_w2h, gas->mlp_theta, gas->mlp_norm};
  const int64_t groups = (n + 31) / 32;
  int blocks = (int)std::min<int64_t>((groups + 3) / 4, (int64_t)sm_count() * 16);
  temperature_mlp_kernel<<<blocks, 128, 0, s>>>(gas->p, n, q, T, iters, m, guess_only, gas->status, mp);
  return cudaGetLastError();
}

cudaError_t mlp_set_params(dg_gas gas, const float* theta_host, const dg_mlp_norm& nrm) {
  cudaError_t e = cudaSuccess;
  if (!gas->mlp_theta) e = cudaMalloc((void**)&gas->mlp_theta, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess)
    e = cudaMemcpy(gas->mlp_theta, theta_host, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ensure_half_weights(gas);
  if (e == cudaSuccess) {
    gas->mlp_norm = nrm;
    gas->has_mlp = true;
  }
  return e;
}

cudaError_t mlp_loss_grad(int64_t n, const float* theta, const float* X, const float* t, float* grad, float* loss,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t blocks = (n + TS - 1) / TS;
  mlp_grad_kernel<<<(unsigned)blocks, TS, kGradSmem, s>>>(theta, X, t, n, 1.0f / (float)n, grad, loss);
  return cudaGetLastError();
}

cudaError_t mlp_train(dg_gas gas, int64_t n, const double* e_dev, const double* Y_dev, const double* T_dev,
                      const dg_mlp_train_opts& o, const float* init_host, float* history) {
  // normalisation from the data (host copies of e and T)
  std::vector<double> he(n), hT(n);
  cudaError_t e = cudaMemcpy(he.data(), e_dev, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hT.data(), T_dev, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  dg_mlp_norm nrm;
  std::memset(&nrm, 0, sizeof(nrm));
  double se = 0, se2 = 0, sT = 0, sT2 = 0, Tmin = hT[0], Tmax = hT[0];
  for (int64_t i = 0; i < n; ++i) {
    se += he[i];
    se2 += he[i] * he[i];
    sT += hT[i];
    sT2 += hT[i] * hT[i];
    Tmin = std::min(Tmin, hT[i]);
    Tmax = std::max(Tmax, hT[i]);
  }
  nrm.e_mean = se / n;
  nrm.e_scale = std::sqrt(std::max(se2 / n - nrm.e_mean * nrm.e_mean, 1e-300));
  nrm.T_mean = sT / n;
  nrm.T_scale = std::sqrt(std::max(sT2 / n - nrm.T_mean * nrm.T_mean, 1e-300));
  nrm.T_min = Tmin;
  nrm.T_max = Tmax;
  float *X = nullptr, *t = nullptr, *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  e = cudaMalloc((void**)&X, sizeof(float) * NI * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&theta, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&grad, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&v, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(theta, init_host, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(grad, 0, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMemset(m, 0, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMemset(v, 0, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) {
    features_kernel<<<sm_count() * 8, 256>>>(n, gas->p.ns, e_dev, Y_dev, T_dev, nrm, X, t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kGradSmem);
  const int64_t batch = o.batch;
  const int64_t nb = n / batch;  // full batches only
  double b1t = 1.0, b2t = 1.0;
  float lr = o.lr;
  for (int ep = 0; ep < o.epochs && e == cudaSuccess; ++ep) {
    e = cudaMemset(loss, 0, sizeof(float));
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
      const int64_t off = ((b + (int64_t)ep * 7919) % nb) * batch;  // batch order rotates per epoch
      mlp_grad_kernel<<<(unsigned)((batch + TS - 1) / TS), TS, kGradSmem>>>(theta, X + off * NI, t + off, batch,
                                                                             1.0f / (float)batch, grad, loss);
      b1t *= 0.9;
      b2t *= 0.999;
      adam_kernel<<<(DG_MLP_PARAMS + 255) / 256, 256>>>(theta, grad, m, v, lr, (float)(1.0 - b1t),
                                                        (float)(1.0 - b2t));
      e = cudaGetLastError();
    }
    float l = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpy(&l, loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (history) history[ep] = l / (float)std::max<int64_t>(nb, 1);
    lr *= o.lr_decay;
  }
  std::vector<float> trained(DG_MLP_PARAMS);
  if (e == cudaSuccess)
    e = cudaMemcpy(trained.data(), theta, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyDeviceToHost);
  cudaFree(X);
  cudaFree(t);
  cudaFree(theta);
  cudaFree(grad);
  cudaFree(m);
  cudaFree(v);
  cudaFree(loss);
  if (e == cudaSuccess) e = mlp_set_params(gas, trained.data(), nrm);
  return e;
}

}  // namespace dg
