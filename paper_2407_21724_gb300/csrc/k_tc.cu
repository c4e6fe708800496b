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
// The near-field product (block-sparse, Eq. 16 blocks) runs through the same
// kernel: pairs (mu, nu) that share a block are one GEMM with the block's real
// form as A (rows (i, re/im) of y_mu, columns (j, re/im) of x_nu) and the
// gathered x_nu rows (FP32 copy of x) as B.  Each pair stores its product to
// its own row of a partials buffer, so all tiles run in one launch, and
// k_near_sum adds a particle's rows in lattice-offset order.
//
// Operands live in shared memory in the K-major 128-byte-swizzled layout:
// rows of 32 FP32 values (128 bytes), 8-row atoms of 1024 bytes, and the
// 16-byte chunk q of row r stored at chunk q ^ (r mod 8).  The coefficient
// images are built in that layout on the host and copied with one bulk copy
// per K chunk; the spectra are gathered, split and swizzled by the threads.
// Every wait is bounded by a polling limit passed to the kernel (the
// context's wait limit).  A wait that runs out sets an error flag; the CTA
// then stops issuing work, waits (with the fixed drain bound TC_SPIN) for
// every bulk copy and MMA commit it has already issued, frees its tensor
// memory and returns, so nothing asynchronous outlives it.
#include <algorithm>
#include <complex>
#include <cstring>

#include "smr_internal.h"

namespace smr {

namespace {

constexpr int TC_NP = 128;                     // particle rows per CTA (MMA N)
constexpr int TC_TILE = 96;                    // particles per tile: 3 waves of smaller tiles on 152 SMs
constexpr int TC_KC = 32;                      // K values per chunk (one swizzle row)
constexpr int TC_ABYTES = 128 * TC_KC * 4;     // one coefficient chunk, one split: 16 KB
constexpr int TC_BBYTES = TC_NP * TC_KC * 4;   // one spectrum chunk, one split: 16 KB
constexpr int TC_STAGE = 2 * TC_ABYTES + 2 * TC_BBYTES;
constexpr int TC_NSTAGE = 3;
constexpr int TC_PF = 3;                       // spectrum chunks of loads in flight per producer
constexpr size_t TC_SMEM = (size_t)TC_NSTAGE * TC_STAGE + 1024 + 2048;   // + alignment, barriers, ids
constexpr uint32_t TC_SPIN = 1u << 24;         // default polling limit; also the drain bound
constexpr int NEAR_NPH = 9;                    // near-product phases: self blocks + 8 lattice offsets

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
// bounded wait: false if the phase did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_test(a, parity)) return true;
  return false;
}
// bounded wait that also gives up as soon as another warp of the CTA has
// raised the abort flag
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t a, uint32_t parity, uint32_t limit,
                                                   volatile int* abort_flag) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_test(a, parity)) return true;
    if (*abort_flag) return false;
  }
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
// A = coefficient images [nK][hi | lo][128 rows][32] (swizzled), one per
// tile (tshape); in0 = B rows [.][K8] (FP32), gathered by perm; y [.][M4]
// (FP64), rows yperm.  Receive: A per shape, in0 the level-0 incoming
// spectra, perm = yperm = particles.  Near: A per block, in0 = x (FP32),
// perm = nu, yperm = mu.
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

template <typename YT>
__global__ void __launch_bounds__(288, 1) k_receive_tc(int nK, int K8, int M4, const int* __restrict__ tshape,
                                                       const int* __restrict__ tstart,
                                                       const int* __restrict__ tcount,
                                                       const int* __restrict__ perm,
                                                       const int* __restrict__ yperm, const float* __restrict__ A,
                                                       const float* __restrict__ in0, YT* __restrict__ y,
                                                       int accumulate, uint32_t spin, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // barriers: fullA[NS] (bulk copy bytes), fullB[NS] (8 producer warps), done[NS] (MMA commit)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TC_NSTAGE * TC_STAGE);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 3 * TC_NSTAGE);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 1);
  int* mus = reinterpret_cast<int*>(slot + 4);                              // [TC_NP] B rows
  int* ys = mus + TC_NP;                                                    // [TC_NP] y rows
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
  if (tid < TC_NP) {
    mus[tid] = tid < cnt ? perm[t0 + tid] : -1;
    ys[tid] = tid < cnt ? yperm[t0 + tid] : -1;
  }
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
          if (!ok && lane == 0) ok = mbar_wait_or_abort(done(st), (use - 1) & 1, spin, abort_flag);
          ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          if (!ok) {
            bad = true;
            *abort_flag = 1;
          } else {
            st_chunk(sm + st * TC_STAGE, tid, r[b]);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fullB(st)) : "memory");
            // the next loads go out after the fence, so it does not wait for them
            if (c + TC_PF < nK) ld_chunk(in0, K8, mus, c + TC_PF, tid, r[b]);
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
    int ncopy = 0;                                   // chunks whose coefficient copy was issued
    for (int c = 0; c < TC_NSTAGE - 1 && c < nK; ++c, ++ncopy) copyA(c);
    int issued = -1;                                 // last chunk whose MMAs were committed
    for (int c = 0; c < nK && !bad; ++c) {
      const int st = c % TC_NSTAGE, use = c / TC_NSTAGE;
      const uint32_t Sa = sm0 + st * TC_STAGE;
      if (!mbar_wait_or_abort(fullA(st), use & 1, spin, abort_flag) ||
          !mbar_wait_or_abort(fullB(st), use & 1, spin, abort_flag)) {
        bad = true;
        break;
      }
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
        if (c >= 1 && !mbar_wait(done((c - 1) % TC_NSTAGE), ((c - 1) / TC_NSTAGE) & 1, spin)) { bad = true; break; }
        copyA(cn);
        ++ncopy;
      }
    }
    // the last commit covers every MMA issued before it
    if (issued >= 0 && !mbar_wait(done(issued % TC_NSTAGE), (issued / TC_NSTAGE) & 1, spin)) bad = true;
    if (issued != nK - 1) bad = true;
    if (bad) {
      *abort_flag = 1;
      // drain: the coefficient copies not yet consumed, then the last commit
      for (int ch = issued + 1; ch < ncopy; ++ch)
        mbar_wait(fullA(ch % TC_NSTAGE), (ch / TC_NSTAGE) & 1, TC_SPIN);
      if (issued >= 0) mbar_wait(done(issued % TC_NSTAGE), (issued / TC_NSTAGE) & 1, TC_SPIN);
    }
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
        if (accumulate) {
          // the 32 columns are distinct y rows: all loads first, then stores
          YT yo[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            int col = g * 32 + j;
            yo[j] = col < cnt ? y[(size_t)ys[col] * M4 + row] : YT(0);
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            int col = g * 32 + j;
            if (col < cnt) y[(size_t)ys[col] * M4 + row] = yo[j] + (YT)v[j];
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            int col = g * 32 + j;
            if (col < cnt) y[(size_t)ys[col] * M4 + row] = (YT)v[j];
          }
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

// Aggregation on the tensor cores (Eq. 26 patterns times coefficients):
//   out0[mu][(direction, field, re/im)] = sum_k' A_s[.][k'] x[mu][k'],
//   k' = (current, mode, re/im) (4 N_psi <= 128: the coefficients of mu).
// A field belongs to one current, so the rows are taken current by current:
// M tile t covers current t & 1 and the rows (direction, component, re/im)
// [128 (t >> 1), 128 (t >> 1) + 128) of it, and reads only that current's
// K chunks (half of K).  Consecutive tiles write the two halves of the same
// output sectors.
// CTA = up to 128 particles of one shape, 288 threads.  The 8 producer
// warps load the tile's coefficients once (FP64 -> split TF32, swizzled,
// resident for the whole CTA) and then drain the accumulators; one control
// thread streams the coefficient images of the M tiles through a bulk-copy
// ring and issues the MMAs into two alternating tensor-memory accumulators,
// so the epilogue of one M tile overlaps the MMAs of the next.
constexpr int AG_NS = 3;                       // coefficient-image stages
constexpr int AG_KCMAX = 4;                    // K chunks (K' <= 128)
constexpr size_t AG_SMEM = (size_t)2 * AG_KCMAX * TC_BBYTES + (size_t)AG_NS * 2 * TC_ABYTES + 1024 + 1024;

template <typename XT>
__global__ void __launch_bounds__(288, 1) k_aggregate_tc(int nMT, int nKc, int K4, int npsi2,
                                                         const int* __restrict__ tshape,
                                                         const int* __restrict__ tstart,
                                                         const int* __restrict__ tcount,
                                                         const int* __restrict__ perm, const float* __restrict__ A,
                                                         const XT* __restrict__ x, float* __restrict__ out0,
                                                         uint32_t spin, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* Bh = reinterpret_cast<float*>(sm);                               // [current][nKc][128][32]
  float* Bl = reinterpret_cast<float*>(sm + AG_KCMAX * TC_BBYTES);
  unsigned char* Ar = sm + 2 * AG_KCMAX * TC_BBYTES;                      // [AG_NS][hi | lo]
  uint64_t* bars = reinterpret_cast<uint64_t*>(Ar + AG_NS * 2 * TC_ABYTES);
  // aFull[NS], aDone[NS], accFull[2], accEmpty[2]
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * AG_NS + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 1);
  int* mus = reinterpret_cast<int*>(slot + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int s = tshape[tile], t0 = tstart[tile], cnt = tcount[tile];
  const uint32_t sm0 = saddr(sm), ar0 = saddr(Ar);
  auto aFull = [&](int st) { return saddr(bars + st); };
  auto aDone = [&](int st) { return saddr(bars + AG_NS + st); };
  auto accFull = [&](int b) { return saddr(bars + 2 * AG_NS + b); };
  auto accEmpty = [&](int b) { return saddr(bars + 2 * AG_NS + 2 + b); };
  const size_t tileA = (size_t)nKc * 2 * 128 * TC_KC;                   // floats per M tile image
  const float* As = A + (size_t)s * nMT * tileA;
  if (warp == 0) tmem_alloc(saddr(slot), 2 * TC_NP);
  if (tid == 0) {
    for (int i = 0; i < AG_NS; ++i) {
      mbar_init(aFull(i), 1);
      mbar_init(aDone(i), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accFull(b), 1);
      mbar_init(accEmpty(b), 8);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (tid < TC_NP) mus[tid] = tid < cnt ? perm[t0 + tid] : -1;
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *slot;
  const int total = nMT * nKc;                        // coefficient chunks in order (M tile, K chunk)
  int ncopy = 0;                                      // chunks whose bulk copy was issued (control thread)
  auto copy_chunk = [&](int g) {
    const int t = g / nKc, c = g % nKc, st = g % AG_NS;
    mbar_expect_tx(aFull(st), 2 * TC_ABYTES);
    bulk_g2s(ar0 + st * 2 * TC_ABYTES, As + t * tileA + (size_t)c * 2 * 128 * TC_KC, 2 * TC_ABYTES, aFull(st));
    ++ncopy;
  };
  if (tid == 288 - 32) {
    // control thread: first coefficient chunks while the producers load x
    for (int g = 0; g < AG_NS - 1 && g < total; ++g) copy_chunk(g);
  }
  if (warp < 8) {
    // the tile's coefficients: row = particle; item = 4 consecutive values of
    // one current's (mode, re/im) run, padded to nKc chunks of 32
    const int per_cur = nKc * 8;                     // items per current and row
    const int ngrp = 128 * 2 * per_cur;
    const int Kx = 2 * npsi2;
    for (int g = tid; g < ngrp; g += 256) {
      const int row = g / (2 * per_cur), rem = g - row * (2 * per_cur);
      const int cur = rem / per_cur, q4 = rem - cur * per_cur;
      const int mu = mus[row], kl = 4 * q4;
      float4 h, l;
      if constexpr (sizeof(XT) == 4) {
        // FP32 copy of x: the split stays on the FP32 units
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (mu >= 0) {
          const float* xr = x + (size_t)mu * Kx + cur * npsi2;
          if (kl + 3 < npsi2) {
            v = *reinterpret_cast<const float4*>(xr + kl);
          } else {
            if (kl < npsi2) v.x = xr[kl];
            if (kl + 1 < npsi2) v.y = xr[kl + 1];
            if (kl + 2 < npsi2) v.z = xr[kl + 2];
          }
        }
        h = make_float4(tf32r(v.x), tf32r(v.y), tf32r(v.z), tf32r(v.w));
        l = make_float4(tf32r(v.x - h.x), tf32r(v.y - h.y), tf32r(v.z - h.z), tf32r(v.w - h.w));
      } else {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (mu >= 0) {
          const double* xr = x + (size_t)mu * Kx + cur * npsi2;
          if (kl + 3 < npsi2) {
            double2 a = *reinterpret_cast<const double2*>(xr + kl), b = *reinterpret_cast<const double2*>(xr + kl + 2);
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
          } else {
            for (int e = 0; e < 4; ++e)
              if (kl + e < npsi2) v[e] = xr[kl + e];
          }
        }
        h.x = tf32r((float)v[0]); l.x = tf32r((float)(v[0] - (double)h.x));
        h.y = tf32r((float)v[1]); l.y = tf32r((float)(v[1] - (double)h.y));
        h.z = tf32r((float)v[2]); l.z = tf32r((float)(v[2] - (double)h.z));
        h.w = tf32r((float)v[3]); l.w = tf32r((float)(v[3] - (double)h.w));
      }
      const int c = cur * nKc + (q4 >> 3), q = q4 & 7;
      const int off = (c * 128 + row) * 32 + ((q ^ (row & 7)) << 2);
      *reinterpret_cast<float4*>(Bh + off) = h;
      *reinterpret_cast<float4*>(Bl + off) = l;
    }
    fence_async_smem();
  }
  __syncthreads();
  bool bad = false;
  if (warp < 8) {
    // ---- epilogue warps: drain the accumulator of each M tile
    const int q4 = warp & 3, half = warp >> 2;
    for (int t = 0; t < nMT && !bad; ++t) {
      const int b = t & 1;
      bool ok = false;
      if (lane == 0) ok = mbar_wait_or_abort(accFull(b), (t >> 1) & 1, spin, abort_flag);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        bad = true;
        *abort_flag = 1;
        break;
      }
      tc_after();
      const int rc = (t >> 1) * 128 + q4 * 32 + lane;   // (direction, component, re/im) of current t & 1
      const int oi = (rc >> 2) * 8 + (t & 1) * 4 + (rc & 3);
#pragma unroll 1
      for (int g = half * 2; g < half * 2 + 2; ++g) {
        if (g * 32 >= cnt) break;                      // uniform per warp
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * TC_NP + g * 32), v);
        if (rc < K4) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            int col = g * 32 + j;
            if (col < cnt) out0[(size_t)mus[col] * (2 * K4) + oi] = v[j];
          }
        }
      }
      tc_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(accEmpty(b)) : "memory");
    }
  } else if (lane == 0) {
    // ---- control thread
    const uint32_t idesc = idesc_tf32(128, TC_NP);
    const uint32_t bh0 = sm0, bl0 = sm0 + AG_KCMAX * TC_BBYTES;
    int g = 0;                                        // next chunk to consume
    uint32_t last_bar = 0, last_par = 0;              // the latest MMA commit (covers all before it)
    bool committed = false;
    for (int t = 0; t < nMT && !bad; ++t) {
      const int b = t & 1;
      if (t >= 2 && !mbar_wait_or_abort(accEmpty(b), ((t >> 1) - 1) & 1, spin, abort_flag)) { bad = true; break; }
      tc_after();
      const uint32_t d = tmem + (uint32_t)(b * TC_NP);
      for (int c = 0; c < nKc; ++c) {
        const int st = g % AG_NS;
        if (!mbar_wait_or_abort(aFull(st), (g / AG_NS) & 1, spin, abort_flag)) { bad = true; break; }
        tc_after();
        const uint32_t Sa = ar0 + st * 2 * TC_ABYTES;
#pragma unroll
        for (int k = 0; k < TC_KC / 8; ++k) {
          uint64_t ah = sdesc_sw128(Sa + 32 * k), al = sdesc_sw128(Sa + TC_ABYTES + 32 * k);
          const int cb = (t & 1) * nKc + c;            // this current's K chunk of the coefficients
          uint64_t bh = sdesc_sw128(bh0 + cb * TC_BBYTES + 32 * k), bl = sdesc_sw128(bl0 + cb * TC_BBYTES + 32 * k);
          mma_tf32(d, ah, bh, idesc, (c > 0 || k > 0) ? 1u : 0u);
          mma_tf32(d, ah, bl, idesc, 1u);
          mma_tf32(d, al, bh, idesc, 1u);
        }
        mma_commit(aDone(st));
        last_bar = aDone(st);
        last_par = (g / AG_NS) & 1;
        committed = true;
        ++g;
        // next coefficient chunk into the stage of chunk g - 2 once its MMAs are done
        const int gn = g - 1 + AG_NS - 1;
        if (gn < total) {
          if (g >= 2 && !mbar_wait(aDone((g - 2) % AG_NS), ((g - 2) / AG_NS) & 1, spin)) { bad = true; break; }
          copy_chunk(gn);
        }
      }
      if (bad) break;
      mma_commit(accFull(b));
      last_bar = accFull(b);
      last_par = (t >> 1) & 1;
    }
    // every MMA is complete once the last M tile's accumulator is full
    if (!bad && nMT > 0 && !mbar_wait(accFull((nMT - 1) & 1), ((nMT - 1) >> 1) & 1, spin)) bad = true;
    if (bad) {
      *abort_flag = 1;
      // drain: the coefficient copies not yet consumed, then the latest commit
      for (int ch = g; ch < ncopy; ++ch) mbar_wait(aFull(ch % AG_NS), (ch / AG_NS) & 1, TC_SPIN);
      if (committed) mbar_wait(last_bar, last_par, TC_SPIN);
    }
  }
  bad = __syncthreads_or(bad) != 0;
  if (bad && tid == 0) atomicExch(err, 1);
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    tmem_dealloc(tmem, 2 * TC_NP);
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
  if (M4 > 128) return SMR_OK;                       // more than one M tile: CUDA-core paths
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
  // aggregation images: row m' = (direction, field, re/im), column k' =
  // (current, mode, re/im); entry = the real form of conj(P(mode, field's
  // component, direction)) where the field's current matches, else 0
  int K4 = 4 * K0, npsi2 = 2 * npsi;
  int nKc = (npsi2 + TC_KC - 1) / TC_KC, nMT = 2 * ((K4 + 127) / 128);
  std::vector<float> agg;
  if (2 * nKc <= AG_KCMAX && npsi % 2 == 0) {
    size_t tileA = (size_t)nKc * 2 * 128 * TC_KC;
    agg.assign((size_t)S * nMT * tileA, 0.f);
    for (int s = 0; s < S; ++s)
      for (int t = 0; t < nMT; ++t)
        for (int rl = 0; rl < 128; ++rl) {
          int rc = (t >> 1) * 128 + rl;
          if (rc >= K4) break;
          int k = rc / 4, comp = (rc / 2) & 1, ro = rc & 1;
          for (int kl = 0; kl < npsi2; ++kl) {
            int n = kl / 2, ri = kl & 1;
            const double2 pv = P[(((size_t)s * npsi + n) * 2 + comp) * K0 + k];
            double v = ro == 0 ? (ri == 0 ? pv.x : pv.y) : (ri == 0 ? -pv.y : pv.x);
            float hi = tf32_host((float)v);
            float lo = tf32_host((float)(v - (double)hi));
            int ch = kl / TC_KC, kk = kl % TC_KC, q = kk >> 2, e = kk & 3;
            size_t base = ((size_t)s * nMT + t) * tileA + (size_t)ch * 2 * 128 * TC_KC;
            size_t off = (size_t)rl * TC_KC + (((q ^ (rl & 7)) << 2) | e);
            agg[base + off] = hi;
            agg[base + (size_t)128 * TC_KC + off] = lo;
          }
        }
  }
  // tiles of up to 128 particles of one shape (particles sorted by shape)
  std::vector<int> perm(c->p), tsh, tst, tcn;
  for (int i = 0; i < c->p; ++i) perm[i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return c->sid[a] < c->sid[b]; });
  for (int i = 0; i < c->p;) {
    int s = c->sid[perm[i]], j = i;
    while (j < c->p && c->sid[perm[j]] == s && j - i < TC_TILE) ++j;
    tsh.push_back(s); tst.push_back(i); tcn.push_back(j - i);
    i = j;
  }
  int rc;
  c->tc_agg_ready = false;
  if (!agg.empty()) {
    if ((rc = upload(c, &c->d_tc_agg, agg))) return rc;
    c->tc_nMT = nMT;
    c->tc_nKc = nKc;
    c->tc_agg_ready = true;
  }
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

// displaced particles take these paths on unshifted per-particle spectra; the
// box sum and broadcast around them apply the shifts
bool tc_receive_ok(const Ctx* c, int R) { return c->tc_enable && c->tc_ready && R == 1; }

int run_receive_tc(Ctx* c, const float2* in0, double2* y, bool accumulate, cudaStream_t st) {
  cudaFuncSetAttribute(k_receive_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  k_receive_tc<double><<<(unsigned)c->tc_ntile, 288, TC_SMEM, st>>>(
      c->tc_nK, 8 * c->lev[0].K, 4 * c->npsi, c->d_tc_shape, c->d_tc_start, c->d_tc_count, c->d_tc_perm,
      c->d_tc_perm, c->d_tc_rec, reinterpret_cast<const float*>(in0), reinterpret_cast<double*>(y), accumulate ? 1 : 0,
      c->tc_spin, c->d_tc_err);
  SMR_LAUNCH(c);
  return SMR_OK;
}

bool tc_aggregate_ok(const Ctx* c, int R) {
  return c->tc_enable && c->tc_ready && c->tc_agg_ready && R == 1;
}

// x32: FP32 copy of x (prep_x32), or null to split the FP64 x
int run_aggregate_tc(Ctx* c, const double2* x, const float2* x32, float2* out0, cudaStream_t st) {
  if (x32) {
    cudaFuncSetAttribute(k_aggregate_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AG_SMEM);
    k_aggregate_tc<float><<<(unsigned)c->tc_ntile, 288, AG_SMEM, st>>>(
        c->tc_nMT, c->tc_nKc, 4 * c->lev[0].K, 2 * c->npsi, c->d_tc_shape, c->d_tc_start, c->d_tc_count,
        c->d_tc_perm, c->d_tc_agg, reinterpret_cast<const float*>(x32), reinterpret_cast<float*>(out0),
        c->tc_spin, c->d_tc_err);
  } else {
    cudaFuncSetAttribute(k_aggregate_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)AG_SMEM);
    k_aggregate_tc<double><<<(unsigned)c->tc_ntile, 288, AG_SMEM, st>>>(
        c->tc_nMT, c->tc_nKc, 4 * c->lev[0].K, 2 * c->npsi, c->d_tc_shape, c->d_tc_start, c->d_tc_count,
        c->d_tc_perm, c->d_tc_agg, reinterpret_cast<const double*>(x), reinterpret_cast<float*>(out0),
        c->tc_spin, c->d_tc_err);
  }
  SMR_LAUNCH(c);
  return SMR_OK;
}

// Near product on the tensor cores.  Block b (n2 x n2 complex, stored
// column-major in d_B64) in real form: row (i, re/im) of y, column (j, re/im)
// of x, entries [Re, -Im; Im, Re] of B_ij; split into TF32 hi / lo and laid
// out like the receive images.  Pairs go to phases by lattice offset (self
// blocks first), and within a phase into tiles of up to TC_NP pairs sharing
// a block.  One launch runs every tile: the pair (mu, nu) of phase ph writes
// its FP32 product to row ph * p + mu of a partials buffer (no two pairs
// share a row, so no read-modify-write), and k_near_sum adds each particle's
// rows in phase order.
int build_near_tc(Ctx* c) {
  c->tcn_ready = false;
  const int n2 = 2 * c->npsi, M4 = 2 * n2, S = c->S, nb = c->nblk;
  if (M4 > 128 || c->p == 0) return SMR_OK;          // more than one M tile: CUDA-core path
  const int nK = (M4 + TC_KC - 1) / TC_KC;
  const size_t bsz = (size_t)n2 * n2;
  std::vector<double2> B((size_t)nb * bsz);
  SMR_CUDA(c, cudaMemcpy(B.data(), c->d_B64, B.size() * sizeof(double2), cudaMemcpyDeviceToHost));
  const size_t per = (size_t)nK * 2 * 128 * TC_KC;
  std::vector<float> img((size_t)nb * per, 0.f);
  for (int b = 0; b < nb; ++b)
    for (int j = 0; j < n2; ++j)
      for (int i = 0; i < n2; ++i) {
        const double2 z = B[(size_t)b * bsz + (size_t)j * n2 + i];
        for (int ro = 0; ro < 2; ++ro)
          for (int ri = 0; ri < 2; ++ri) {
            const int row = 2 * i + ro, kp = 2 * j + ri;
            const double v = ro == 0 ? (ri == 0 ? z.x : -z.y) : (ri == 0 ? z.y : z.x);
            const float hi = tf32_host((float)v), lo = tf32_host((float)(v - (double)hi));
            const int ch = kp / TC_KC, kk = kp % TC_KC, q = kk >> 2, e = kk & 3;
            const size_t base = (size_t)b * per + (size_t)ch * 2 * 128 * TC_KC;
            const size_t off = (size_t)row * TC_KC + (((q ^ (row & 7)) << 2) | e);
            img[base + off] = hi;
            img[base + (size_t)128 * TC_KC + off] = lo;
          }
      }
  // phase of a block: 0 for self blocks, 1..8 for the lattice offsets
  auto phase_of = [&](int b) {
    if (b < S) return 0;
    const int o = (c->blk_dy[b] + 1) * 3 + (c->blk_dx[b] + 1);
    return o < 4 ? o + 1 : o;
  };
  const int NPH = NEAR_NPH;
  std::vector<std::vector<int>> pr(NPH);               // pair indices e per phase
  std::vector<int> emu(c->nr_col.size());
  std::vector<unsigned short> seen((size_t)c->p * NPH, 0);
  for (int mu = 0; mu < c->p; ++mu)
    for (int e = c->nr_ptr[mu]; e < c->nr_ptr[mu + 1]; ++e) {
      const int b = c->nr_blk[e];
      const int dx = b < S ? 0 : c->blk_dx[b], dy = b < S ? 0 : c->blk_dy[b];
      if (dx < -1 || dx > 1 || dy < -1 || dy > 1) return SMR_OK;   // not a lattice neighbour
      if (b >= S && dx == 0 && dy == 0) return SMR_OK;
      const int ph = phase_of(b);
      seen[(size_t)mu * NPH + ph]++;
      emu[e] = mu;
      pr[ph].push_back(e);
    }
  // each y row at most once per phase (no two CTAs of a launch write it),
  // and exactly once in phase 0, which writes instead of adding
  for (int mu = 0; mu < c->p; ++mu)
    for (int ph = 0; ph < NPH; ++ph)
      if (seen[(size_t)mu * NPH + ph] > 1 || (ph == 0 && seen[(size_t)mu * NPH] != 1)) return SMR_OK;
  std::vector<int> tb, ts, tn, pnu, pmu, phase(1, 0);
  std::vector<unsigned short> pmask(c->p, 0);             // phases in which each particle has a pair
  for (int mu = 0; mu < c->p; ++mu)
    for (int ph = 0; ph < NPH; ++ph)
      if (seen[(size_t)mu * NPH + ph]) pmask[mu] |= (unsigned short)(1u << ph);
  std::vector<double> bytes, flops;
  for (int ph = 0; ph < NPH; ++ph) {
    std::vector<int>& v = pr[ph];
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return c->nr_blk[a] < c->nr_blk[b]; });
    std::vector<char> used(nb, 0);
    int nbu = 0;
    for (size_t i = 0; i < v.size();) {
      const int b = c->nr_blk[v[i]];
      size_t j = i;
      while (j < v.size() && c->nr_blk[v[j]] == b && j - i < (size_t)TC_NP) ++j;
      tb.push_back(b);
      ts.push_back((int)pnu.size());
      tn.push_back((int)(j - i));
      for (size_t k = i; k < j; ++k) {
        const int e = v[k];
        pnu.push_back(c->nr_col[e]);
        pmu.push_back(ph * c->p + emu[e]);
      }
      if (!used[b]) { used[b] = 1; ++nbu; }
      i = j;
    }
    phase.push_back((int)tb.size());
    const double np = (double)v.size();
    // x row (FP32) read, partial row (FP32) written, each block once
    bytes.push_back(np * M4 * (4.0 + 4.0) + (double)nbu * bsz * 8.0);
    flops.push_back(8.0 * (double)bsz * np);
  }
  int rc;
  if ((rc = upload(c, &c->d_tcn_img, img)) || (rc = upload(c, &c->d_tcn_blk, tb)) ||
      (rc = upload(c, &c->d_tcn_start, ts)) || (rc = upload(c, &c->d_tcn_count, tn)) ||
      (rc = upload(c, &c->d_tcn_nu, pnu)) || (rc = upload(c, &c->d_tcn_mu, pmu)) ||
      (rc = upload(c, &c->d_tcn_mask, pmask)))
    return rc;
  if (c->d_tcn_part) cudaFree(c->d_tcn_part);
  c->d_tcn_part = nullptr;
  c->tcn_part_bytes = (size_t)NPH * c->p * M4 * sizeof(float);
  SMR_CUDA(c, cudaMalloc((void**)&c->d_tcn_part, c->tcn_part_bytes));
  if (c->d_x32) cudaFree(c->d_x32);
  c->d_x32 = nullptr;
  SMR_CUDA(c, cudaMalloc((void**)&c->d_x32, (size_t)c->p * n2 * sizeof(float2)));
  if (!c->d_tc_err) SMR_CUDA(c, cudaMalloc((void**)&c->d_tc_err, sizeof(int)));
  c->tcn_nK = nK;
  c->tcn_phase = phase;
  c->tcn_bytes = bytes;
  c->tcn_flops = flops;
  c->tcn_ready = true;
  return SMR_OK;
}

bool tc_near_ok(const Ctx* c, int R) { return c->tc_enable && c->tcn_ready && R == 1; }

// y[mu][r] = sum over the phases in which mu has a pair, in phase order, of
// the partial rows (FP32).  Thread = 4 consecutive r; the present phases'
// loads are all issued before the sums.
__global__ void k_near_sum(int p, int M44, const unsigned short* __restrict__ mask,
                           const float4* __restrict__ part, double2* __restrict__ y) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p * M44) return;
  const int mu = (int)(t / M44), r4 = (int)(t - (long long)mu * M44);
  const unsigned m = mask[mu];
  float4 v[NEAR_NPH];
#pragma unroll
  for (int ph = 0; ph < NEAR_NPH; ++ph)
    v[ph] = (m >> ph & 1u) ? part[((size_t)ph * p + mu) * M44 + r4] : make_float4(0.f, 0.f, 0.f, 0.f);
  // FP32 sums (FP64 adds and conversions run at 1/64 of the FP32 rate here;
  // the CUDA-core near kernel accumulates in FP32 too)
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int ph = 0; ph < NEAR_NPH; ++ph)
    if (m >> ph & 1u) {
      a.x += v[ph].x;
      a.y += v[ph].y;
      a.z += v[ph].z;
      a.w += v[ph].w;
    }
  y[2 * t] = make_double2(a.x, a.y);
  y[2 * t + 1] = make_double2(a.z, a.w);
}

// x must already be in d_x32 (prep_x32)
int run_near_tc(Ctx* c, double2* y, cudaStream_t st) {
  const int n2 = 2 * c->npsi, M4 = 2 * n2;
  const int nt = c->tcn_phase.back();
  double bytes = 0, flops = 0;
  for (size_t ph = 0; ph < c->tcn_bytes.size(); ++ph) {
    bytes += c->tcn_bytes[ph];
    flops += c->tcn_flops[ph];
  }
  cudaFuncSetAttribute(k_receive_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  pbeg(c, st, "near", -1, bytes, flops);
  k_receive_tc<float><<<(unsigned)nt, 288, TC_SMEM, st>>>(
      c->tcn_nK, M4, M4, c->d_tcn_blk, c->d_tcn_start, c->d_tcn_count, c->d_tcn_nu, c->d_tcn_mu,
      c->d_tcn_img, reinterpret_cast<const float*>(c->d_x32), c->d_tcn_part, 0, c->tc_spin, c->d_tc_err);
  SMR_LAUNCH(c);
  pend(c, st);
  const long long nm = (long long)c->p * M4, nt4 = nm / 4;
  pbeg(c, st, "near", -1, (double)nm * 8.0 + (double)c->nr_col.size() * M4 * 4.0 + 2.0 * c->p, 0.0);
  k_near_sum<<<(unsigned)((nt4 + 255) / 256), 256, 0, st>>>(c->p, M4 / 4, c->d_tcn_mask,
                                                           reinterpret_cast<const float4*>(c->d_tcn_part), y);
  SMR_LAUNCH(c);
  pend(c, st);
  return SMR_OK;
}

// 0 = no failed wait seen since the last check (clears the flag)
int tc_check(Ctx* c) {
  if (!c->d_tc_err) return SMR_OK;
  int h = 0;
  SMR_CUDA(c, cudaMemcpy(&h, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(c->d_tc_err, 0, sizeof(int));
    c->err = "tensor-core product step: a pipeline wait ran out (results of that product are invalid)";
    return SMR_E_TIMEOUT;
  }
  return SMR_OK;
}

}  // namespace smr
