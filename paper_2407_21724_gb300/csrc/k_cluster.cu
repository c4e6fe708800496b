// Cluster block-Jacobi preconditioner (not in the paper; an option next to
// its block-diagonal one, Sec. V stage v): the particles are grouped into
// 2 x 2 lattice clusters (the quadtree's level-1 boxes of each array), and
// the preconditioner applies, per cluster, the inverse of the cluster's part
// of the near-field matrix: the self blocks and the near blocks between the
// cluster's members (every pair in a 2 x 2 cluster is a lattice neighbour).
//
// Set-up on the GPU in FP64, in batches of clusters: the cluster matrix
// (4 m x 4 m, m = 2 n_psi; an absent member's rows and columns are the
// identity) is assembled from the stored near blocks, inverted in place by
// Gauss-Jordan elimination with partial pivoting (one CTA per cluster), and
// stored transposed, in FP64 and FP32, so that the apply kernel's threads
// (one per output row) read consecutive addresses.
#include <cmath>
#include <map>
#include <tuple>

#include "smr_internal.h"

namespace smr {

namespace {

__device__ inline double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// A[b] (N x N row-major, N = 4 m) for the clusters [c0, c0 + nb): member a's
// rows against member b's columns from the near block (mem_a, mem_b); the
// blocks are stored transposed, Bt[col * m + row].
__global__ void k_cluster_assemble(int c0, int nb, int m, const int* __restrict__ mem,
                                   const int* __restrict__ ptr, const int* __restrict__ col,
                                   const int* __restrict__ blk, const double2* __restrict__ Bt,
                                   double2* __restrict__ A) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  const int cl = c0 + b;
  const int N = 4 * m;
  __shared__ int bid[16];
  if (threadIdx.x < 16) {
    const int a = threadIdx.x / 4, bb = threadIdx.x % 4;
    const int pa = mem[4 * cl + a], pb = mem[4 * cl + bb];
    int id = -1;
    if (pa >= 0 && pb >= 0)
      for (int k = ptr[pa]; k < ptr[pa + 1]; ++k)
        if (col[k] == pb) id = blk[k];
    bid[threadIdx.x] = id;
  }
  __syncthreads();
  double2* Ab = A + (size_t)b * N * N;
  for (long long idx = threadIdx.x; idx < (long long)N * N; idx += blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const int a = i / m, bb = j / m, ii = i % m, jj = j % m;
    const int id = bid[4 * a + bb];
    double2 v = make_double2(0.0, 0.0);
    if (id >= 0) v = Bt[(size_t)id * m * m + (size_t)jj * m + ii];
    else if (i == j && mem[4 * cl + a] < 0) v = make_double2(1.0, 0.0);
    Ab[idx] = v;
  }
}

// In-place Gauss-Jordan inversion with partial pivoting of A[b] (N x N), one
// CTA per matrix; then the inverse, transposed, into out64 / out32 slot c0+b.
// A zero pivot sets *bad and leaves the slot's inverse zero.
__global__ void __launch_bounds__(256) k_cluster_invert(int c0, int nb, int N, double2* __restrict__ A,
                                                        double2* __restrict__ out64, float2* __restrict__ out32,
                                                        int* __restrict__ bad) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  double2* M = A + (size_t)b * N * N;
  extern __shared__ double2 colk[];          // [N] column k before the elimination
  __shared__ int piv[1024];
  __shared__ double rv[256];
  __shared__ int ri[256];
  __shared__ int singular;
  if (threadIdx.x == 0) singular = 0;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    // pivot: the largest |M[i][k]| for i >= k
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
      const double2 v = M[(size_t)i * N + k];
      const double mag = v.x * v.x + v.y * v.y;
      if (mag > best) { best = mag; bi = i; }
    }
    rv[threadIdx.x] = best;
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const double o = rv[threadIdx.x + s];
        const int oi = ri[threadIdx.x + s];
        if (o > rv[threadIdx.x] || (o == rv[threadIdx.x] && oi < ri[threadIdx.x])) {
          rv[threadIdx.x] = o;
          ri[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const int p = ri[0];
    if (threadIdx.x == 0) {
      piv[k] = p;
      if (!(rv[0] > 0.0)) singular = 1;
    }
    __syncthreads();
    if (singular) break;
    if (p != k)
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const double2 t = M[(size_t)k * N + j];
        M[(size_t)k * N + j] = M[(size_t)p * N + j];
        M[(size_t)p * N + j] = t;
      }
    __syncthreads();
    const double2 pv = M[(size_t)k * N + k];
    const double d = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = make_double2(pv.x / d, -pv.y / d);
    for (int i = threadIdx.x; i < N; i += blockDim.x) colk[i] = M[(size_t)i * N + k];
    __syncthreads();
    // row k scaled by 1/pivot, its pivot entry replaced by 1/pivot
    for (int j = threadIdx.x; j < N; j += blockDim.x)
      M[(size_t)k * N + j] = (j == k) ? inv : cmul2(M[(size_t)k * N + j], inv);
    __syncthreads();
    for (long long idx = threadIdx.x; idx < (long long)N * N; idx += blockDim.x) {
      const int i = (int)(idx / N), j = (int)(idx % N);
      if (i == k) continue;
      const double2 f = colk[i];
      const double2 rk = M[(size_t)k * N + j];
      if (j == k) {
        M[idx] = make_double2(-(f.x * rk.x - f.y * rk.y), -(f.x * rk.y + f.y * rk.x));
      } else {
        double2 v = M[idx];
        v.x -= f.x * rk.x - f.y * rk.y;
        v.y -= f.x * rk.y + f.y * rk.x;
        M[idx] = v;
      }
    }
    __syncthreads();
  }
  if (singular) {
    if (threadIdx.x == 0) atomicExch(bad, 1);
    for (long long idx = threadIdx.x; idx < (long long)N * N; idx += blockDim.x) {
      out64[(size_t)(c0 + b) * N * N + idx] = make_double2(0.0, 0.0);
      out32[(size_t)(c0 + b) * N * N + idx] = make_float2(0.f, 0.f);
    }
    return;
  }
  // undo the row exchanges as column exchanges, in reverse order
  for (int k = N - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 t = M[(size_t)i * N + k];
        M[(size_t)i * N + k] = M[(size_t)i * N + p];
        M[(size_t)i * N + p] = t;
      }
    __syncthreads();
  }
  // transposed copies: out[j][i] = inverse[i][j]
  for (long long idx = threadIdx.x; idx < (long long)N * N; idx += blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx % N);
    const double2 v = M[(size_t)i * N + j];
    out64[(size_t)(c0 + b) * N * N + idx] = v;
    out32[(size_t)(c0 + b) * N * N + idx] = make_float2((float)v.x, (float)v.y);
  }
}

// z = (cluster inverse) r for one cluster and right-hand side per CTA: the
// cluster's rows of r staged in shared memory, one output row per thread.
template <typename V>
__global__ void k_cluster_apply(int m, int R, const int* __restrict__ mem, const V* __restrict__ AinvT,
                                const double2* __restrict__ r, double2* __restrict__ z) {
  const int cl = blockIdx.x / R, rr = blockIdx.x % R;
  const int N = 4 * m;
  extern __shared__ double2 xs[];
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int p = mem[4 * cl + j / m];
    xs[j] = p >= 0 ? r[((size_t)p * m + j % m) * R + rr] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const V* Ab = AinvT + (size_t)cl * N * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int p = mem[4 * cl + i / m];
    if (p < 0) continue;
    double ax = 0, ay = 0;
    if (sizeof(V) == sizeof(float2)) {
      float fx = 0.f, fy = 0.f;
      for (int j = 0; j < N; ++j) {
        const float2 a = reinterpret_cast<const float2*>(Ab)[(size_t)j * N + i];
        const float bx = (float)xs[j].x, by = (float)xs[j].y;
        fx = fmaf(a.x, bx, fmaf(-a.y, by, fx));
        fy = fmaf(a.x, by, fmaf(a.y, bx, fy));
      }
      ax = fx;
      ay = fy;
    } else {
      for (int j = 0; j < N; ++j) {
        const double2 a = reinterpret_cast<const double2*>(Ab)[(size_t)j * N + i];
        ax += a.x * xs[j].x - a.y * xs[j].y;
        ay += a.x * xs[j].y + a.y * xs[j].x;
      }
    }
    z[((size_t)p * m + i % m) * R + rr] = make_double2(ax, ay);
  }
}

}  // namespace

bool cluster_ok(const Ctx* c) { return 8 * c->npsi <= 256; }

int build_clusters(Ctx* c) {
  if (c->cl_ready) return SMR_OK;
  if (c->multi) {
    c->err = "the cluster preconditioner needs at most one particle per lattice cell";
    return SMR_E_INVALID_ARG;
  }
  if (!cluster_ok(c)) {
    c->err = "the cluster preconditioner needs 4 x 2 n_psi <= 256 (n_psi <= 32)";
    return SMR_E_INVALID_ARG;
  }
  const int m = 2 * c->npsi, N = 4 * m;
  // clusters: (array, floor(i/2), floor(j/2)) of each particle's lattice cell
  std::map<std::tuple<int, int, int>, int> key;
  std::vector<int> mem;
  for (int p = 0; p < c->p; ++p) {
    const int ci = c->pi[p] >= 0 ? c->pi[p] / 2 : -((-c->pi[p] + 1) / 2);
    const int cj = c->pj[p] >= 0 ? c->pj[p] / 2 : -((-c->pj[p] + 1) / 2);
    auto it = key.emplace(std::make_tuple(c->arr.empty() ? 0 : c->arr[p], ci, cj), (int)key.size());
    const int cl = it.first->second;
    if (it.second) mem.insert(mem.end(), {-1, -1, -1, -1});
    const int slot = (((c->pi[p] % 2) + 2) % 2) * 2 + (((c->pj[p] % 2) + 2) % 2);
    mem[4 * cl + slot] = p;
  }
  const int ncl = (int)key.size();
  int* d_mem = nullptr;
  SMR_CUDA(c, cudaMalloc((void**)&d_mem, mem.size() * sizeof(int)));
  SMR_CUDA(c, cudaMemcpy(d_mem, mem.data(), mem.size() * sizeof(int), cudaMemcpyHostToDevice));
  const size_t nn = (size_t)N * N;
  double2* inv64 = nullptr;
  float2* inv32 = nullptr;
  const int batch = std::max(1, std::min(ncl, 2048));
  double2* scratch = nullptr;
  int* d_bad = nullptr;
  bool ok = cudaMalloc((void**)&inv64, (size_t)ncl * nn * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&inv32, (size_t)ncl * nn * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&scratch, (size_t)batch * nn * sizeof(double2)) == cudaSuccess &&
            cudaMalloc((void**)&d_bad, sizeof(int)) == cudaSuccess;
  auto release = [&]() {
    cudaFree(scratch);
    cudaFree(d_bad);
  };
  if (!ok) {
    cudaGetLastError();
    release();
    cudaFree(inv64);
    cudaFree(inv32);
    cudaFree(d_mem);
    c->err = "out of device memory for the cluster preconditioner";
    return SMR_E_OOM;
  }
  cudaMemset(d_bad, 0, sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(k_cluster_invert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(N * sizeof(double2)));
  for (int c0 = 0; c0 < ncl && e == cudaSuccess; c0 += batch) {
    const int nb = std::min(batch, ncl - c0);
    k_cluster_assemble<<<nb, 256>>>(c0, nb, m, d_mem, c->d_nr_ptr, c->d_nr_col, c->d_nr_blk, c->d_B64, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
    k_cluster_invert<<<nb, 256, N * sizeof(double2)>>>(c0, nb, N, scratch, inv64, inv32, d_bad);
    e = cudaGetLastError();
  }
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
  release();
  if (e != cudaSuccess) {
    cudaFree(inv64);
    cudaFree(inv32);
    cudaFree(d_mem);
    c->err = std::string("cluster preconditioner set-up: ") + cudaGetErrorString(e);
    return SMR_E_CUDA;
  }
  if (bad) {
    cudaFree(inv64);
    cudaFree(inv32);
    cudaFree(d_mem);
    c->err = "a cluster's near-field matrix is singular: the cluster preconditioner is undefined";
    return SMR_E_INVALID_ARG;
  }
  c->ncl = ncl;
  c->d_cl_mem = d_mem;
  c->d_cl_inv64 = inv64;
  c->d_cl_inv32 = inv32;
  c->cl_ready = true;
  return SMR_OK;
}

int run_cluster(Ctx* c, int R, int prec, const double2* r, double2* z, cudaStream_t st) {
  if (!c->cl_ready) {
    c->err = "cluster preconditioner not built";
    return SMR_E_STATE;
  }
  const int m = 2 * c->npsi, N = 4 * m;
  const int threads = std::min(256, N);
  const size_t sm = (size_t)N * sizeof(double2);
  if (prec == SMR_PREC_FP64)
    k_cluster_apply<double2><<<(unsigned)(c->ncl * R), threads, sm, st>>>(m, R, c->d_cl_mem, c->d_cl_inv64, r, z);
  else
    k_cluster_apply<float2><<<(unsigned)(c->ncl * R), threads, sm, st>>>(m, R, c->d_cl_mem, c->d_cl_inv32, r, z);
  SMR_CUDA(c, cudaGetLastError());
  return SMR_OK;
}

void free_clusters(Ctx* c) {
  cudaFree(c->d_cl_mem);
  cudaFree(c->d_cl_inv64);
  cudaFree(c->d_cl_inv32);
  c->d_cl_mem = nullptr;
  c->d_cl_inv64 = nullptr;
  c->d_cl_inv32 = nullptr;
  c->ncl = 0;
  c->cl_ready = false;
}

}  // namespace smr
