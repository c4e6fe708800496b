// Dense per-shape contractions of the FP32 product on the 5th-generation
// tensor cores (tcgen05 MMA, accumulators in tensor memory).
//
// Receive (Eqs. 24-25) with the combination of the four incoming fields
// folded into a per-shape coefficient matrix is a real GEMM
//   y[mu][m'] += sum_k' A_s[m'][k'] B[mu][k'],
//   m' = (current, mode, re/im)          (4 N_psi <= 128 rows: one MMA M tile)
//   k' = (direction, field, re/im)       (8 K_0: the level-0 incoming spectrum
//                                          of particle mu, contiguous in HBM)
// with particles of one shape as the N dimension.  FP32 accuracy comes from
// split TF32: a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi), and
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs per K step, FP32
// accumulation in tensor memory).
//
// Operands live in shared memory in the K-major 128-byte-swizzled layout:
// rows of 32 FP32 values (128 bytes), 8-row atoms of 1024 bytes, and the
// 16-byte chunk q of row r stored at chunk q ^ (r mod 8).  The coefficient
// images are built in that layout on the host and copied with one bulk copy
// per K chunk; the spectra are gathered, split and swizzled by the threads.
// Every wait is bounded; a wait that runs out sets an error flag, the CTA
// stops issuing work, frees its tensor memory and returns.
#include <algorithm>
#include <complex>
#include <cstring>

#include "smr_internal.h"

namespace smr {

namespace {

constexpr int TC_NP = 128;                     // particles per CTA (MMA N)
constexpr int TC_KC = 32;                      // K values per chunk (one swizzle row)
constexpr int TC_ABYTES = 128 * TC_KC * 4;     // one coefficient chunk, one split: 16 KB
constexpr int TC_BBYTES = TC_NP * TC_KC * 4;   // one spectrum chunk, one split: 16 KB
constexpr int TC_STAGE = 2 * TC_ABYTES + 2 * TC_BBYTES;
constexpr int TC_NSTAGE = 3;
constexpr int TC_PF = 3;                       // spectrum chunks of loads in flight per producer
constexpr size_t TC_SMEM = (size_t)TC_NSTAGE * TC_STAGE + 1024 + 1024;   // + alignment, barriers, ids
constexpr uint32_t TC_SPIN = 1u << 24;         // try_wait rounds before giving up

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major operand, 128-byte swizzle: start >> 4, leading offset 16 B (unused
// for this layout), stride between 8-row atoms 1024 B, descriptor version 1,
// swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t a) {
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32, both K-major.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the phase did not complete
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  for (uint32_t i = 0; i < TC_SPIN; ++i)
    if (mbar_test(a, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t t, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 consecutive columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t t, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(t));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Receive on the tensor cores: CTA = up to 128 particles of one shape, 256
// threads.  K runs in chunks of 32 through a ring of TC_NSTAGE shared-memory
// stages: the coefficient chunk arrives by one bulk copy issued a chunk ahead;
// the spectrum chunk (128 rows x 128 bytes, read 4 rows per warp instruction)
// is loaded two chunks ahead into registers, then split into TF32 hi / lo and
// stored swizzled.  Thread 0 issues the 12 MMAs of a chunk (4 K steps x 3
// products) and commits them to the stage's barrier.
// A = per-shape coefficient images [nK][hi | lo][128 rows][32] (swizzled),
// in0 = level-0 incoming spectra [p][K8] (FP32), y [p][M4] (FP64).
__device__ __forceinline__ void ld_chunk(const float* __restrict__ in0, int K8, const int* mus, int c, int tid,
                                         float4* r) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int idx = tid + 256 * j, row = idx >> 3, q = idx & 7;
    int mu = mus[row], kk = c * TC_KC + 4 * q;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mu >= 0) {
      const float* b = in0 + (size_t)mu * K8 + kk;
      if (kk + 3 < K8) {
        v = *reinterpret_cast<const float4*>(b);
      } else {
        if (kk < K8) v.x = b[0];
        if (kk + 1 < K8) v.y = b[1];
        if (kk + 2 < K8) v.z = b[2];
      }
    }
    r[j] = v;
  }
}

__device__ __forceinline__ void st_chunk(unsigned char* S, int tid, const float4* r) {
  float* Bh = reinterpret_cast<float*>(S + 2 * TC_ABYTES);
  float* Bl = reinterpret_cast<float*>(S + 2 * TC_ABYTES + TC_BBYTES);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int idx = tid + 256 * j, row = idx >> 3, q = idx & 7;
    float4 v = r[j];
    float4 h = make_float4(tf32r(v.x), tf32r(v.y), tf32r(v.z), tf32r(v.w));
    float4 l = make_float4(tf32r(v.x - h.x), tf32r(v.y - h.y), tf32r(v.z - h.z), tf32r(v.w - h.w));
    int off = row * 32 + ((q ^ (row & 7)) << 2);
    *reinterpret_cast<float4*>(Bh + off) = h;
    *reinterpret_cast<float4*>(Bl + off) = l;
  }
}

__global__ void __launch_bounds__(288, 1) k_receive_tc(int nK, int K8, int M4, const int* __restrict__ tshape,
                                                       const int* __restrict__ tstart,
                                                       const int* __restrict__ tcount,
                                                       const int* __restrict__ perm, const float* __restrict__ A,
                                                       const float* __restrict__ in0, double* __restrict__ y,
                                                       int accumulate, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // barriers: fullA[NS] (bulk copy bytes), fullB[NS] (8 producer warps), done[NS] (MMA commit)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TC_NSTAGE * TC_STAGE);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3 * TC_NSTAGE);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 1);
  int* mus = reinterpret_cast<int*>(slot + 4);                              // [TC_NP]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int s = tshape[tile], t0 = tstart[tile], cnt = tcount[tile];
  const uint32_t sm0 = saddr(sm);
  auto fullA = [&](int st) { return saddr(bars + st); };
  auto fullB = [&](int st) { return saddr(bars + TC_NSTAGE + st); };
  auto done = [&](int st) { return saddr(bars + 2 * TC_NSTAGE + st); };
  const float* As = A + (size_t)s * nK * (2 * 128 * TC_KC);
  if (warp == 0) tmem_alloc(saddr(slot), TC_NP);
  if (tid == 0) {
    for (int i = 0; i < TC_NSTAGE; ++i) {
      mbar_init(fullA(i), 1);
      mbar_init(fullB(i), 8);
      mbar_init(done(i), 1);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (tid < TC_NP) mus[tid] = tid < cnt ? perm[t0 + tid] : -1;
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *slot;
  bool bad = false;
  if (warp < 8) {
    // ---- producers: spectrum chunks, TC_PF chunks of loads in flight (the
    // loop is unrolled by TC_PF so that each register buffer is only read a
    // full round after its loads were issued)
    float4 r[TC_PF][4];
#pragma unroll
    for (int b = 0; b < TC_PF; ++b)
      if (b < nK) ld_chunk(in0, K8, mus, b, tid, r[b]);
#pragma unroll 1
    for (int cb = 0; cb < nK && !bad; cb += TC_PF) {
#pragma unroll
      for (int b = 0; b < TC_PF; ++b) {
        const int c = cb + b;
        if (c < nK && !bad) {
          const int st = c % TC_NSTAGE, use = c / TC_NSTAGE;
          // lane 0 waits for the stage; the outcome is shared so the warp
          // takes one path (the arrive below needs all 32 lanes)
          bool ok = c < TC_NSTAGE;
          if (!ok && lane == 0) {
            for (uint32_t i = 0; i < TC_SPIN && !ok; ++i) {
              ok = mbar_test(done(st), (use - 1) & 1);
              if (!ok && *abort_flag) break;
            }
          }
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok) {
            bad = true;
            *abort_flag = 1;
          } else {
            st_chunk(sm + st * TC_STAGE, tid, r[b]);
            if (c + TC_PF < nK) ld_chunk(in0, K8, mus, c + TC_PF, tid, r[b]);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fullB(st)) : "memory");
          }
        }
      }
    }
  } else if (lane == 0) {
    // ---- control thread: coefficient copies ahead of use, MMAs, commits
    const uint32_t idesc = idesc_tf32(128, TC_NP);
    auto copyA = [&](int c) {
      const int st = c % TC_NSTAGE;
      mbar_expect_tx(fullA(st), 2 * TC_ABYTES);
      bulk_g2s(sm0 + st * TC_STAGE, As + (size_t)c * (2 * 128 * TC_KC), 2 * TC_ABYTES, fullA(st));
    };
    for (int c = 0; c < TC_NSTAGE - 1 && c < nK; ++c) copyA(c);
    int issued = -1;
    for (int c = 0; c < nK && !bad; ++c) {
      const int st = c % TC_NSTAGE, use = c / TC_NSTAGE;
      const uint32_t Sa = sm0 + st * TC_STAGE;
      bool ok = false;
      for (uint32_t i = 0; i < TC_SPIN && !ok; ++i) {
        ok = mbar_test(fullA(st), use & 1) && mbar_test(fullB(st), use & 1);
        if (!ok && *abort_flag) break;
      }
      if (!ok) { bad = true; break; }
      tc_after();
#pragma unroll
      for (int k = 0; k < TC_KC / 8; ++k) {
        uint64_t ah = sdesc_sw128(Sa + 32 * k), al = sdesc_sw128(Sa + TC_ABYTES + 32 * k);
        uint64_t bh = sdesc_sw128(Sa + 2 * TC_ABYTES + 32 * k);
        uint64_t bl = sdesc_sw128(Sa + 2 * TC_ABYTES + TC_BBYTES + 32 * k);
        mma_tf32(tmem, ah, bh, idesc, (c > 0 || k > 0) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      mma_commit(done(st));
      issued = c;
      // coefficients of chunk c + NS - 1 go to the stage of chunk c - 1 once its MMAs are done
      const int cn = c + TC_NSTAGE - 1;
      if (cn < nK) {
        if (c >= 1 && !mbar_wait(done((c - 1) % TC_NSTAGE), ((c - 1) / TC_NSTAGE) & 1)) { bad = true; break; }
        copyA(cn);
      }
    }
    // the last commit covers every MMA issued before it
    if (issued >= 0 && !mbar_wait(done(issued % TC_NSTAGE), (issued / TC_NSTAGE) & 1)) bad = true;
    if (issued != nK - 1) bad = true;
    if (bad) *abort_flag = 1;
  }
  bad = __syncthreads_or(bad) != 0;
  if (!bad && warp < 8) {
    tc_after();
    const int q4 = warp & 3, half = warp >> 2;         // lane quarter, column half
    const int row = q4 * 32 + lane;                    // m'
#pragma unroll 1
    for (int g = half * 2; g < half * 2 + 2; ++g) {
      if (g * 32 >= cnt) break;                        // uniform per warp
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(g * 32), v);
      if (row < M4) {
        // the 32 columns are distinct particles: all loads first, then stores
        double yo[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          int col = g * 32 + j;
          yo[j] = (accumulate && col < cnt) ? y[(size_t)mus[col] * M4 + row] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          int col = g * 32 + j;
          if (col < cnt) y[(size_t)mus[col] * M4 + row] = yo[j] + (double)v[j];
        }
      }
    }
  } else if (bad && tid == 0) {
    atomicExch(err, 1);
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_dealloc(tmem, TC_NP);
  }
}

// TF32 rounding on the host (round to nearest, ties away), for the split
float tf32_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

// Coefficient images of the tensor-core receive for every shape, from the
// FP64 patterns: row m' = (current, mode, re/im), column k' = (direction,
// field, re/im); entry = the real form of -j k w_k c(current, field) P(mode,
// field's component, k), c from Eqs. 24-25 (zeta B0 + B3, zeta B1 - B2,
// -B1 + B2/zeta, B0 + B3/zeta for the electric rows and the magnetic ones).
int build_tc(Ctx* c) {
  c->tc_ready = false;
  Level& L0 = c->lev[0];
  int npsi = c->npsi, K0 = L0.K, S = c->S;
  int M4 = 4 * npsi, K8 = 8 * K0;
  if (M4 > 128) return SMR_OK;                       // more than one M tile: CUDA-core receive
  int nK = (K8 + TC_KC - 1) / TC_KC;
  size_t nP = (size_t)S * npsi * 2 * K0;
  std::vector<double2> P(nP);
  SMR_CUDA(c, cudaMemcpy(P.data(), c->d_P64, nP * sizeof(double2), cudaMemcpyDeviceToHost));
  std::vector<float> img((size_t)S * nK * 2 * 128 * TC_KC, 0.f);
  typedef std::complex<double> cx;
  const cx mjk(0.0, -c->k);
  const double z = c->zeta, iz = 1.0 / c->zeta;
  for (int s = 0; s < S; ++s)
    for (int row = 0; row < M4; ++row) {
      int cur = row / (2 * npsi), m = (row / 2) % npsi, ro = row & 1;
      for (int kp = 0; kp < K8; ++kp) {
        int k = kp / 8, f = (kp / 2) & 3, ri = kp & 1;
        const double2 pt = P[(((size_t)s * npsi + m) * 2 + 0) * K0 + k];
        const double2 pp = P[(((size_t)s * npsi + m) * 2 + 1) * K0 + k];
        cx Pt(pt.x, pt.y), Pp(pp.x, pp.y), cf;
        if (cur == 0) cf = f == 0 ? z * Pt : f == 1 ? z * Pp : f == 2 ? -Pp : Pt;
        else cf = f == 0 ? Pp : f == 1 ? -Pt : f == 2 ? iz * Pt : iz * Pp;
        cf *= mjk * L0.w[k];
        double v = ro == 0 ? (ri == 0 ? cf.real() : -cf.imag()) : (ri == 0 ? cf.imag() : cf.real());
        float hi = tf32_host((float)v);
        float lo = tf32_host((float)(v - (double)hi));
        int ch = kp / TC_KC, kk = kp % TC_KC, q = kk >> 2, e = kk & 3;
        size_t base = (((size_t)s * nK + ch) * 2) * 128 * TC_KC;
        size_t off = (size_t)row * TC_KC + (((q ^ (row & 7)) << 2) | e);
        img[base + off] = hi;
        img[base + (size_t)128 * TC_KC + off] = lo;
      }
    }
  // tiles of up to 128 particles of one shape (particles sorted by shape)
  std::vector<int> perm(c->p), tsh, tst, tcn;
  for (int i = 0; i < c->p; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return c->sid[a] < c->sid[b]; });
  for (int i = 0; i < c->p;) {
    int s = c->sid[perm[i]], j = i;
    while (j < c->p && c->sid[perm[j]] == s && j - i < TC_NP) ++j;
    tsh.push_back(s); tst.push_back(i); tcn.push_back(j - i);
    i = j;
  }
  int rc;
  if ((rc = upload(c, &c->d_tc_rec, img)) || (rc = upload(c, &c->d_tc_perm, perm)) ||
      (rc = upload(c, &c->d_tc_shape, tsh)) || (rc = upload(c, &c->d_tc_start, tst)) ||
      (rc = upload(c, &c->d_tc_count, tcn)))
    return rc;
  if (!c->d_tc_err) SMR_CUDA(c, cudaMalloc((void**)&c->d_tc_err, sizeof(int)));
  SMR_CUDA(c, cudaMemset(c->d_tc_err, 0, sizeof(int)));
  c->tc_nK = nK;
  c->tc_ntile = (int)tsh.size();
  c->tc_ready = true;
  return SMR_OK;
}

bool tc_receive_ok(const Ctx* c, int R) { return c->tc_enable && c->tc_ready && R == 1 && !c->any_dshift; }

int run_receive_tc(Ctx* c, const float2* in0, double2* y, bool accumulate, cudaStream_t st) {
  cudaFuncSetAttribute(k_receive_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  k_receive_tc<<<(unsigned)c->tc_ntile, 288, TC_SMEM, st>>>(
      c->tc_nK, 8 * c->lev[0].K, 4 * c->npsi, c->d_tc_shape, c->d_tc_start, c->d_tc_count, c->d_tc_perm,
      c->d_tc_rec, reinterpret_cast<const float*>(in0), reinterpret_cast<double*>(y), accumulate ? 1 : 0,
      c->d_tc_err);
  SMR_LAUNCH(c);
  return SMR_OK;
}

// 0 = no failed wait seen since the last check (clears the flag)
int tc_check(Ctx* c) {
  if (!c->d_tc_err) return SMR_OK;
  int h = 0;
  SMR_CUDA(c, cudaMemcpy(&h, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(c->d_tc_err, 0, sizeof(int));
    c->err = "tensor-core receive: a pipeline wait ran out (results of that product are invalid)";
    return SMR_E_CUDA;
  }
  return SMR_OK;
}

}  // namespace smr
