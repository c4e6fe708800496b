// Learned initial guess for the GMRES solve: per-scatterer features, a 4-layer
// MLP (BF16 weights, FP32 activations and accumulation, FP32 Adam master
// weights) trained on solutions of the plain solver, and the re-phasing that
// turns its output into coefficients.
//
// Features of particle mu (F = 448):
//   for each of the 48 lattice neighbours within 2 wavelengths (0 < dx^2+dy^2 <= 16
//   cells at pitch 0.5, fixed order by distance then angle): one-hot shape (8)
//   and presence (1); own shape one-hot (8); incidence direction (3) and the
//   real polarisation vector (3); 2 zeros of padding.
// Output (O = 4 n_psi): real and imaginary parts of the de-phased coefficients
//   abar_mu = alpha_mu exp(+j k khat . r_mu) / scale, [Re(e,m modes) | Im(e,m modes)].
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "smr_internal.h"

namespace smr {

namespace {

constexpr int kSlots = 48;
constexpr int kShapesMax = 8;

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[M x N] = op(A)[M x K] op(B)[K x N], FP32 accumulation.
//   A(m, k) = TRA ? A[row(k) * lda + m] : A[row(m) * lda + k],  row(r) = aidx ? aidx[r] : r
//   B(k, n) = TRB ? B[n * ldb + k]      : B[k * ldb + n]
template <typename TA, typename TB, bool TRA, bool TRB>
__global__ void k_gemm(int M, int N, int K, const TA* __restrict__ A, int lda, const int* __restrict__ aidx,
                       const TB* __restrict__ B, int ldb, float* __restrict__ C, int ldc) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int t = threadIdx.x; t < 64 * 16; t += 256) {
      int mm = t % 64, kk = t / 64;           // A tile element (m, k)
      int m = m0 + mm, k = k0 + kk;
      float va = 0.f;
      if (m < M && k < K) {
        if (TRA) va = ld(A + (size_t)(aidx ? aidx[k] : k) * lda + m);
        else va = ld(A + (size_t)(aidx ? aidx[m] : m) * lda + k);
      }
      As[kk][mm] = va;
      int nn = t % 64;                         // B tile element (k, n)
      int n = n0 + nn;
      float vb = 0.f;
      if (n < N && k < K) vb = TRB ? ld(B + (size_t)n * ldb + k) : ld(B + (size_t)k * ldb + n);
      Bs[kk][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) C[(size_t)m * ldc + n] = acc[i][j];
    }
}

template <typename TA, typename TB, bool TRA, bool TRB>
int gemm(Ctx* c, int M, int N, int K, const TA* A, int lda, const int* aidx, const TB* B, int ldb, float* C,
         int ldc, cudaStream_t st) {
  dim3 g((N + 63) / 64, (M + 63) / 64);
  k_gemm<TA, TB, TRA, TRB><<<g, 256, 0, st>>>(M, N, K, A, lda, aidx, B, ldb, C, ldc);
  SMR_LAUNCH(c);
  return SMR_OK;
}

// Z += bias (per column); A = silu(Z) when act
__global__ void k_bias_act(int n, int w, float* __restrict__ Z, const float* __restrict__ bias,
                           float* __restrict__ A, int act) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * w) return;
  float z = Z[t] + bias[t % w];
  Z[t] = z;
  if (act) A[t] = silu(z);
}

// dZ = dA * silu'(Z)
__global__ void k_act_back(long long n, const float* __restrict__ Z, const float* __restrict__ dA,
                           float* __restrict__ dZ) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) dZ[t] = dA[t] * dsilu(Z[t]);
}

// db[j] = sum_m dZ[m][j]
__global__ void k_colsum(int M, int N, const float* __restrict__ dZ, float* __restrict__ db) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dZ[(size_t)m * N + j];
  db[j] = s;
}

// mean squared error: dY = 2 (Y - T) / (n O); per-block partial sums of (Y - T)^2
__global__ void k_mse(int n, int O, const float* __restrict__ Y, const float* __restrict__ T,
                      const int* __restrict__ tidx, float* __restrict__ dY, double* __restrict__ part) {
  __shared__ double red[256];
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (t < (long long)n * O) {
    int m = (int)(t / O), o = (int)(t % O);
    int row = tidx ? tidx[m] : m;
    float d = Y[t] - T[(size_t)row * O + o];
    dY[t] = 2.f * d / ((float)n * (float)O);
    e2 = (double)d * d;
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum(int n, const double* __restrict__ part, double scale, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s * scale;
  }
}

__global__ void k_adam(long long n, float* __restrict__ p, __nv_bfloat16* __restrict__ w16,
                       const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, float lr,
                       float b1, float b2, float eps, float bc1, float bc2) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  float gt = g[t];
  float mt = b1 * m[t] + (1.f - b1) * gt;
  float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  float pt = p[t] - lr * (mt / bc1) / (sqrtf(vt / bc2) + eps);
  p[t] = pt;
  w16[t] = __float2bfloat16(pt);
}

__global__ void k_to_bf16(long long n, const float* __restrict__ p, __nv_bfloat16* __restrict__ w16) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) w16[t] = __float2bfloat16(p[t]);
}

// features, one thread per particle
__global__ void k_features(int p, int F, const int* __restrict__ sid, const int* __restrict__ arr,
                           const int* __restrict__ pi, const int* __restrict__ pj, int map_x0, int map_y0,
                           int map_w, int map_h, const int* __restrict__ boxmap, const int* __restrict__ slots,
                           const double* __restrict__ khat, const double* __restrict__ pol,
                           float* __restrict__ feat) {
  int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= p) return;
  float* f = feat + (size_t)mu * F;
  for (int i = 0; i < F; ++i) f[i] = 0.f;
  for (int s = 0; s < kSlots; ++s) {
    int x = pi[mu] + slots[2 * s] - map_x0, y = pj[mu] + slots[2 * s + 1] - map_y0;
    if (x < 0 || y < 0 || x >= map_w || y >= map_h) continue;
    int nu = boxmap[y * map_w + x];
    if (nu < 0) continue;
    f[s * 9 + sid[nu]] = 1.f;
    f[s * 9 + 8] = 1.f;
  }
  f[kSlots * 9 + sid[mu]] = 1.f;
  int a = arr[mu];
  for (int d = 0; d < 3; ++d) {
    f[kSlots * 9 + 8 + d] = (float)khat[3 * a + d];
    f[kSlots * 9 + 11 + d] = (float)pol[6 * a + 2 * d];
  }
}

// targets: de-phased coefficients / scale
__global__ void k_targets(int p, int npsi, const int* __restrict__ arr, const double* __restrict__ cen,
                          const double* __restrict__ khat, const double2* __restrict__ x, double kw,
                          double inv_scale, float* __restrict__ tgt) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int n2 = 2 * npsi;
  if (t >= (long long)p * n2) return;
  int mu = (int)(t / n2), i = (int)(t % n2);
  const double* kh = khat + 3 * arr[mu];
  const double* r = cen + 3 * mu;
  double sn, cs;
  sincos(kw * (kh[0] * r[0] + kh[1] * r[1] + kh[2] * r[2]), &sn, &cs);
  double2 v = x[(size_t)mu * n2 + i];
  tgt[(size_t)mu * 2 * n2 + i] = (float)((v.x * cs - v.y * sn) * inv_scale);
  tgt[(size_t)mu * 2 * n2 + n2 + i] = (float)((v.x * sn + v.y * cs) * inv_scale);
}

// re-phase the network output into coefficients x0
__global__ void k_rephase(int p, int npsi, int row0, int rows, const int* __restrict__ arr,
                          const double* __restrict__ cen, const double* __restrict__ khat,
                          const float* __restrict__ Y, double kw, double scale, double2* __restrict__ x0) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int n2 = 2 * npsi;
  if (t >= (long long)rows * n2) return;
  int m = (int)(t / n2), i = (int)(t % n2);
  int mu = row0 + m;
  const double* kh = khat + 3 * arr[mu];
  const double* r = cen + 3 * mu;
  double sn, cs;
  sincos(-kw * (kh[0] * r[0] + kh[1] * r[1] + kh[2] * r[2]), &sn, &cs);
  double re = scale * Y[(size_t)m * 2 * n2 + i], im = scale * Y[(size_t)m * 2 * n2 + n2 + i];
  x0[(size_t)mu * n2 + i] = make_double2(re * cs - im * sn, re * sn + im * cs);
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

long long woff(const NN& nn, int l) {
  long long o = 0;
  for (int q = 0; q < l; ++q) o += (long long)nn.dims[q] * nn.dims[q + 1] + nn.dims[q + 1];
  return o;
}

}  // namespace

void nn_free(Ctx* c) {
  NN& nn = c->nn;
  cudaFree(nn.p32); cudaFree(nn.w16); cudaFree(nn.m); cudaFree(nn.v); cudaFree(nn.g);
  cudaFree(nn.act); cudaFree(nn.dact); cudaFree(nn.d_loss); cudaFree(nn.d_slots);
  nn = NN();
}

int nn_init(Ctx* c, int width, unsigned long long seed) {
  if (c->npsi <= 0) { c->err = "set the scene before smr_nn_init (output size is 4 n_psi)"; return SMR_E_STATE; }
  if (width < 1 || width > 4096) { c->err = "width must be in 1..4096"; return SMR_E_INVALID_ARG; }
  nn_free(c);
  NN& nn = c->nn;
  nn.H = width;
  nn.O = 4 * c->npsi;
  int dims[5] = {nn.F, width, width, width, nn.O};
  for (int i = 0; i < 5; ++i) nn.dims[i] = dims[i];
  nn.np = woff(nn, 4);
  std::vector<float> p((size_t)nn.np, 0.f);
  uint64_t s = seed;
  for (int l = 0; l < 4; ++l) {
    long long o = woff(nn, l);
    double a = std::sqrt(6.0 / (nn.dims[l] + nn.dims[l + 1]));
    for (long long i = 0; i < (long long)nn.dims[l] * nn.dims[l + 1]; ++i) {
      double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
      p[o + i] = (float)((2.0 * u - 1.0) * a);
    }
  }
  nn.cap = 8192;
  size_t abytes = (size_t)nn.cap * (6 * (size_t)width + nn.O) * sizeof(float);
  SMR_CUDA(c, cudaMalloc((void**)&nn.p32, nn.np * sizeof(float)));
  SMR_CUDA(c, cudaMalloc((void**)&nn.w16, nn.np * sizeof(__nv_bfloat16)));
  SMR_CUDA(c, cudaMalloc((void**)&nn.m, nn.np * sizeof(float)));
  SMR_CUDA(c, cudaMalloc((void**)&nn.v, nn.np * sizeof(float)));
  SMR_CUDA(c, cudaMalloc((void**)&nn.g, nn.np * sizeof(float)));
  SMR_CUDA(c, cudaMalloc((void**)&nn.act, abytes));
  SMR_CUDA(c, cudaMalloc((void**)&nn.dact, abytes + (size_t)nn.cap * nn.F * sizeof(float)));
  SMR_CUDA(c, cudaMalloc((void**)&nn.d_loss, ((size_t)nn.cap * nn.O / 256 + 2) * sizeof(double)));
  SMR_CUDA(c, cudaMemcpy(nn.p32, p.data(), nn.np * sizeof(float), cudaMemcpyHostToDevice));
  SMR_CUDA(c, cudaMemset(nn.m, 0, nn.np * sizeof(float)));
  SMR_CUDA(c, cudaMemset(nn.v, 0, nn.np * sizeof(float)));
  k_to_bf16<<<(unsigned)((nn.np + 255) / 256), 256>>>(nn.np, nn.p32, nn.w16);
  SMR_LAUNCH(c);
  // neighbour slots within 2 wavelengths, by distance then angle
  std::vector<std::pair<std::pair<int, double>, std::pair<int, int>>> sl;
  for (int dy = -4; dy <= 4; ++dy)
    for (int dx = -4; dx <= 4; ++dx) {
      int d2 = dx * dx + dy * dy;
      if (d2 == 0 || d2 > 16) continue;
      sl.push_back({{d2, std::atan2((double)dy, (double)dx)}, {dx, dy}});
    }
  std::sort(sl.begin(), sl.end());
  std::vector<int> slots;
  for (auto& e : sl) { slots.push_back(e.second.first); slots.push_back(e.second.second); }
  int rc = upload(c, &nn.d_slots, slots);
  if (rc) return rc;
  SMR_CUDA(c, cudaDeviceSynchronize());
  return SMR_OK;
}

int nn_features(Ctx* c, const double* d_khat, const double* d_pol, float* feat, cudaStream_t st) {
  if (!c->nn.p32) { c->err = "call smr_nn_init first"; return SMR_E_STATE; }
  if (c->S > kShapesMax) { c->err = "learned features support at most 8 shapes"; return SMR_E_INVALID_ARG; }
  if (c->multi) { c->err = "learned features need at most one particle per lattice cell"; return SMR_E_INVALID_ARG; }
  Level& L0 = c->lev[0];
  // lattice indices of particles (level-0 boxes are the particles)
  int* d_pi = nullptr;
  int* d_pj = nullptr;
  int rc;
  if ((rc = upload(c, &d_pi, c->pi)) || (rc = upload(c, &d_pj, c->pj))) return rc;
  k_features<<<(c->p + 127) / 128, 128, 0, st>>>(c->p, c->nn.F, c->d_sid, c->d_arr, d_pi, d_pj, L0.map_x0,
                                                  L0.map_y0, L0.map_w, L0.map_h, L0.d_boxmap, c->nn.d_slots,
                                                  d_khat, d_pol, feat);
  SMR_LAUNCH(c);
  SMR_CUDA(c, cudaStreamSynchronize(st));
  cudaFree(d_pi);
  cudaFree(d_pj);
  return SMR_OK;
}

int nn_targets(Ctx* c, const double* d_khat, const double2* x, double scale, float* tgt, cudaStream_t st) {
  long long n = (long long)c->p * 2 * c->npsi;
  k_targets<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c->p, c->npsi, c->d_arr, c->d_centres, d_khat, x, c->k,
                                                         1.0 / scale, tgt);
  SMR_LAUNCH(c);
  return SMR_OK;
}

// Forward (and backward into nn.g) over n rows of feat (rows idx[] if given).
int nn_forward_backward(Ctx* c, int n, const float* feat, const int* idx, const float* tgt, bool backward,
                        double* loss_host, cudaStream_t st) {
  NN& nn = c->nn;
  if (!nn.p32) { c->err = "call smr_nn_init first"; return SMR_E_STATE; }
  if (n < 1 || n > nn.cap) { c->err = "batch must be 1..8192 rows"; return SMR_E_INVALID_ARG; }
  int H = nn.H, O = nn.O;
  // activation layout: Z1 A1 Z2 A2 Z3 A3 Y
  float* Z[4];
  float* A[4];
  Z[0] = nn.act;
  A[0] = Z[0] + (size_t)nn.cap * H;
  Z[1] = A[0] + (size_t)nn.cap * H;
  A[1] = Z[1] + (size_t)nn.cap * H;
  Z[2] = A[1] + (size_t)nn.cap * H;
  A[2] = Z[2] + (size_t)nn.cap * H;
  Z[3] = A[2] + (size_t)nn.cap * H;   // output Y [n][O]
  int rc;
  for (int l = 0; l < 4; ++l) {
    int in = nn.dims[l], out = nn.dims[l + 1];
    const __nv_bfloat16* W = nn.w16 + woff(nn, l);
    const float* b = nn.p32 + woff(nn, l) + (long long)in * out;
    if (l == 0) rc = gemm<float, __nv_bfloat16, false, false>(c, n, out, in, feat, in, idx, W, out, Z[0], out, st);
    else rc = gemm<float, __nv_bfloat16, false, false>(c, n, out, in, A[l - 1], in, nullptr, W, out, Z[l], out, st);
    if (rc) return rc;
    k_bias_act<<<(unsigned)(((long long)n * out + 255) / 256), 256, 0, st>>>(n, out, Z[l], b, l < 3 ? A[l] : nullptr,
                                                                          l < 3 ? 1 : 0);
    SMR_LAUNCH(c);
  }
  // loss and dY
  float* dZ[4];
  float* dA = nn.dact;                         // [cap][max(F, H)]
  dZ[3] = dA + (size_t)nn.cap * std::max(nn.F, H);
  dZ[2] = dZ[3] + (size_t)nn.cap * O;
  dZ[1] = dZ[2] + (size_t)nn.cap * H;
  dZ[0] = dZ[1] + (size_t)nn.cap * H;
  if (!tgt) return SMR_OK;                      // inference only
  int nb = (int)(((long long)n * O + 255) / 256);
  k_mse<<<nb, 256, 0, st>>>(n, O, Z[3], tgt, idx, dZ[3], nn.d_loss + 1);
  SMR_LAUNCH(c);
  k_sum<<<1, 32, 0, st>>>(nb, nn.d_loss + 1, 1.0 / ((double)n * O), nn.d_loss);
  SMR_LAUNCH(c);
  if (backward) {
    for (int l = 3; l >= 0; --l) {
      int in = nn.dims[l], out = nn.dims[l + 1];
      float* gW = nn.g + woff(nn, l);
      float* gb = gW + (long long)in * out;
      const float* Ain = l == 0 ? feat : A[l - 1];
      const int* ai = l == 0 ? idx : nullptr;
      // dW = A_in^T dZ
      rc = gemm<float, float, true, false>(c, in, out, n, Ain, in, ai, dZ[l], out, gW, out, st);
      if (rc) return rc;
      k_colsum<<<(out + 127) / 128, 128, 0, st>>>(n, out, dZ[l], gb);
      SMR_LAUNCH(c);
      if (l > 0) {
        // dA_{l-1} = dZ_l W_l^T ; dZ_{l-1} = dA * silu'(Z_{l-1})
        const __nv_bfloat16* W = nn.w16 + woff(nn, l);
        rc = gemm<float, __nv_bfloat16, false, true>(c, n, in, out, dZ[l], out, nullptr, W, out, dA, in, st);
        if (rc) return rc;
        long long ne = (long long)n * in;
        k_act_back<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(ne, Z[l - 1], dA, dZ[l - 1]);
        SMR_LAUNCH(c);
      }
    }
  }
  if (loss_host) {
    SMR_CUDA(c, cudaMemcpyAsync(loss_host, nn.d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    SMR_CUDA(c, cudaStreamSynchronize(st));
  }
  return SMR_OK;
}

int nn_adam(Ctx* c, float lr, cudaStream_t st) {
  NN& nn = c->nn;
  nn.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  float bc1 = 1.f - std::pow(b1, (float)nn.step), bc2 = 1.f - std::pow(b2, (float)nn.step);
  k_adam<<<(unsigned)((nn.np + 255) / 256), 256, 0, st>>>(nn.np, nn.p32, nn.w16, nn.g, nn.m, nn.v, lr, b1, b2,
                                                         1e-8f, bc1, bc2);
  SMR_LAUNCH(c);
  return SMR_OK;
}

int nn_predict(Ctx* c, const double* d_khat, const double* d_pol, double scale, double2* x0, cudaStream_t st) {
  NN& nn = c->nn;
  float* feat = nullptr;
  SMR_CUDA(c, cudaMalloc((void**)&feat, (size_t)c->p * nn.F * sizeof(float)));
  int rc = nn_features(c, d_khat, d_pol, feat, st);
  for (int r0 = 0; rc == SMR_OK && r0 < c->p; r0 += nn.cap) {
    int rows = std::min(nn.cap, c->p - r0);
    rc = nn_forward_backward(c, rows, feat + (size_t)r0 * nn.F, nullptr, nullptr, false, nullptr, st);
    if (rc) break;
    float* Y = nn.act + (size_t)6 * nn.cap * nn.H;
    long long ne = (long long)rows * 2 * c->npsi;
    k_rephase<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(c->p, c->npsi, r0, rows, c->d_arr, c->d_centres, d_khat,
                                                           Y, c->k, scale, x0);
    SMR_LAUNCH(c);
  }
  cudaStreamSynchronize(st);
  cudaFree(feat);
  return rc;
}

// Learned local-coupling preconditioner: per unknown, the ratio of the
// network's predicted coefficient to the isolated-particle response
// (blockdiag(Z_s^-1) b), with its magnitude clamped to [0.1, 10] (a zero or
// undefined ratio becomes 0.1).
__global__ void k_lpc_ratio(long long n, const double2* __restrict__ xp, const double2* __restrict__ zi,
                            double2* __restrict__ D) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 a = xp[i], b = zi[i];
  double bb = b.x * b.x + b.y * b.y;
  double2 r = make_double2(0.0, 0.0);
  if (bb > 0) r = make_double2((a.x * b.x + a.y * b.y) / bb, (a.y * b.x - a.x * b.y) / bb);
  double m = sqrt(r.x * r.x + r.y * r.y);
  if (!(m > 0.1)) {
    r = (m > 0) ? make_double2(0.1 * r.x / m, 0.1 * r.y / m) : make_double2(0.1, 0.0);
  } else if (m > 10.0) {
    r = make_double2(10.0 * r.x / m, 10.0 * r.y / m);
  }
  D[i] = r;
}

// z[i] *= D[i]
__global__ void k_lpc_apply(long long n, const double2* __restrict__ D, double2* __restrict__ z) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 d = D[i], v = z[i];
  z[i] = make_double2(d.x * v.x - d.y * v.y, d.x * v.y + d.y * v.x);
}

int nn_precond(Ctx* c, const double* d_khat, const double* d_pol, double scale, const double2* b, cudaStream_t st) {
  long long n = 2LL * c->npsi * c->p;
  double2 *xp = nullptr, *zi = nullptr;
  if (!c->d_lpc) SMR_CUDA(c, cudaMalloc((void**)&c->d_lpc, n * sizeof(double2)));
  SMR_CUDA(c, cudaMalloc((void**)&xp, n * sizeof(double2)));
  if (cudaMalloc((void**)&zi, n * sizeof(double2)) != cudaSuccess) {
    cudaFree(xp);
    c->err = "out of device memory";
    return SMR_E_OOM;
  }
  int rc = nn_predict(c, d_khat, d_pol, scale, xp, st);
  if (!rc) rc = run_precond(c, 1, SMR_PREC_FP64, b, zi, st);
  if (!rc) {
    k_lpc_ratio<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, xp, zi, c->d_lpc);
    if (cudaGetLastError() != cudaSuccess) { c->err = "lpc kernel launch"; rc = SMR_E_CUDA; }
  }
  cudaStreamSynchronize(st);
  cudaFree(xp);
  cudaFree(zi);
  c->lpc_ready = (rc == SMR_OK);
  return rc;
}

int lpc_apply(Ctx* c, double2* z, cudaStream_t st) {
  long long n = 2LL * c->npsi * c->p;
  k_lpc_apply<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, c->d_lpc, z);
  SMR_LAUNCH(c);
  return SMR_OK;
}

}  // namespace smr
