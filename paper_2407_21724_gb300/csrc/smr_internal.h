// Internal declarations of libsmr: context, per-level tables, kernel launchers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/smr.h"

namespace smr {

typedef std::complex<double> cd;

// ------------------------------------------------------------------ host math
namespace hm {
// n-point Gauss-Legendre rule on [-1,1], nodes descending (theta ascending).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
// Real orthonormal Y_lm (m >= 0, kind 0 = cos, 1 = sin) and its surface
// gradient components dY/dtheta, (1/sin theta) dY/dphi.
void real_ylm(int l, int m, int kind, double theta, double phi, double* Y, double* Yt, double* Yp);
// Spherical Bessel j_l, y_l for l = 0..L at real x > 0 (Miller downward for j,
// upward for y).
void sph_bessel(int L, double x, std::vector<double>& j, std::vector<double>& y);
// Riccati psi_l(x) = x j_l, xi_l(x) = x h^(2)_l and derivatives.
void riccati(int l, double x, double* psi, double* dpsi, cd* xi, cd* dxi);
// In-place inverse of an n x n complex row-major matrix (partial pivoting).
bool invert(int n, std::vector<cd>& a);
// Modes of a sphere shell list: (l, m, kind) for the first n modes.
void mode_list(int n, std::vector<int>& l, std::vector<int>& m, std::vector<int>& kind);
}  // namespace hm

// ------------------------------------------------------------------ data
// Static modes of a meshed shape (smr_add_shape_mesh): the mode -> RWG
// matrix of Eq. 20, the kept eigenvalues, the geometry, per triangle and
// mode the affine field psi = alpha r - beta ([nt][n_psi][alpha, beta xyz]),
// and the 3-point samples handed to the solver like a sampled shape.
struct MeshModes {
  int ne = 0, nt = 0, nq = 0;
  std::vector<double> M, gamma;
  std::vector<double> geo_V;
  std::vector<int> geo_T;
  std::vector<double> area, nrm, ab;
  std::vector<double> rq, modes;
};

struct Shape {
  double a;                               // sphere radius, or bounding radius of a sampled shape
  int n_perp, n_par;
  int n_psi() const { return n_perp + n_par; }
  // shape given as data (smr_add_shape_sampled): points and weights [nq][4],
  // mode fields and divergences [n_psi][nq][4], self block [2n][2n]
  bool sampled = false;
  int nq = 0;
  std::vector<double> rq, modes;
  std::vector<cd> Z;
  // meshed shape: the self block is assembled for the scene's media
  bool mesh = false;
  MeshModes mm;
  double lateral = 0;                     // largest distance of a point from the z axis
  // rotated copy of another shape (about the z axis): the shape whose self
  // block it shares (rotation leaves Z_s unchanged), -1 if none
  int rot_base = -1;
  double rot_angle = 0;
};

struct Level {
  int L = 0, K = 0, nth = 0, nph = 0, nbox = 0;
  double box = 0;
  std::vector<double> khat, w;          // [K][3], [K]
  std::vector<int> bi, bj;               // box integer coordinates
  std::vector<double> centre;            // [nbox][3]
  std::vector<int> il_ptr, il_src, il_off;  // interaction list CSR by target box
  std::vector<int> off_dx, off_dy;       // unique offsets (box units)
  std::vector<int> parent, quad;         // to level s+1
  std::vector<int> ch_ptr, ch_idx, ch_quad;  // children at level s-1 (s >= 1)
  // device
  double* d_khat = nullptr;
  double* d_w = nullptr;
  int* d_il_ptr = nullptr;
  int* d_il_src = nullptr;
  int* d_il_off = nullptr;
  int* d_il_pk = nullptr;                // [n_il] source box * 64 + table row (few-box kernel)
  double2* d_T64 = nullptr;              // [noff][K]
  float2* d_T32 = nullptr;
  int* d_parent = nullptr;
  int* d_quad = nullptr;
  float2* d_shift4_32 = nullptr;   // [K][4] the four quadrants' shifts per direction (parent level's child tables)
  int* d_ch_ptr = nullptr;
  int* d_ch_idx = nullptr;
  int* d_ch_quad = nullptr;
  // interpolation from this level (child) to s+1 (parent) -- stored on the child
  int* d_th_src = nullptr;               // [nth_p][4] source theta row
  int* d_th_refl = nullptr;              // [nth_p][4] 1 if reflected through a pole
  double* d_th_w64 = nullptr;            // [nth_p][4]
  float* d_th_w32 = nullptr;
  int* d_th_pk = nullptr;                 // [nth_parent][4] source row | reflected << 16
  double* d_th_ws64 = nullptr;            // [nth_parent][4] weights, reflection sign folded in
  float* d_th_ws32 = nullptr;
  int* d_ph_src = nullptr;               // [nph_p][4]
  double* d_ph_w64 = nullptr;
  float* d_ph_w32 = nullptr;
  double2* d_shift64 = nullptr;          // [4][K_p] exp(j k khat_p.(c_c - c_p))
  float2* d_shift32 = nullptr;
  // separable passes (stored on the child level):
  int* d_tht_ptr = nullptr;              // [nth+1] theta-transposed taps by child row
  int* d_tht_tp = nullptr;               //   parent row
  int* d_tht_refl = nullptr;             //   1 if reflected through a pole
  double* d_tht_w64 = nullptr;           //   sign x weight / w_theta(child row)
  float* d_tht_w32 = nullptr;
  int* d_pht_ptr = nullptr;              // [nph+1] phi-transposed taps by child column
  int* d_pht_jp = nullptr;               //   parent column
  double* d_pht_w64 = nullptr;           //   weight x dphi_p / dphi_c
  float* d_pht_w32 = nullptr;
  double* d_wthp64 = nullptr;            // [nth_p] parent theta weights
  float* d_wthp32 = nullptr;
  // dense lattice map of the boxes of this level (translation tiles)
  int map_x0 = 0, map_y0 = 0, map_w = 0, map_h = 0;
  int* d_boxmap = nullptr;               // [map_h][map_w] box index or -1
  int* d_offid = nullptr;                // [7][7] offset (dx+3, dy+3) -> table row or -1
  int ntile_x = 0, ntile_y = 0, ntile_ne = 0;
  int* d_tiles = nullptr;                // non-empty 4x4 translation tiles (ty * ntile_x + tx)
  int ntile8_x = 0, ntile8_ne = 0;
  int* d_tiles8 = nullptr;               // non-empty 8x8 tiles (single right-hand side kernel)
  // fused single right-hand-side anterpolation into this level: child theta
  // rows in nit tiles of TI, parent rows [lo, hi) per tile ([2][nit]), GR the
  // widest range, JC the column chunk per precision (FP64, FP32)
  int ant_TI = 0, ant_nit = 0, ant_GR = 0;
  int ant_JC[2] = {0, 0};
  int ant_JC5 = 0;                       // column chunk of the per-parent FP32 kernel (four quadrants' rows)
  int* d_ant_lo = nullptr;
  // the transposed taps padded to fixed widths (multiples of 4, zero weights):
  // phi by child column [nph][PM] (parent column, weight x dphi_p / dphi_c),
  // theta by child row [nth][TM] (parent row | refl << 16, sign x weight / w_theta)
  // launch variants chosen by smr_autotune per precision (FP64, FP32), one
  // right-hand side; 0 = the built-in rule.  Translation: 1 / 2 = 8x8 target
  // tiles with the full / half direction chunk, 3 = 4x4 tiles, 4 = the
  // few-box kernel (threads along the directions).  Interpolation
  // into the parent of this level: 0 = the built-in rule (the staged kernel
  // k_interp2 in FP32 where its tile fits), 1 = k_interp1 with the full, 2 =
  // with half the theta-row tile.
  int tune_tr[2] = {0, 0};
  int tune_ip[2] = {0, 0};
  // anterpolation into this level: 0 = the built-in rule (k_anterp1), 1 =
  // k_anterp1 with half the column chunk, 2 = with 256 threads, 4 = the
  // staged kernel k_anterp2 (FP32, where its tile fits)
  int tune_an[2] = {0, 0};
  // staged single right-hand-side FP32 interpolation into the parent of this
  // level (k_interp2): tiles of ip2_TR parent theta rows, each with the band
  // of child rows [first, first + count) its theta taps read ([2][nrt]);
  // ip2_BR the widest band; ip2_NCP / ip2_RPT the phi-pass shape (column
  // parts and rows per thread)
  int ip2_TR = 0, ip2_nrt = 0, ip2_BR = 0, ip2_NCP = 0, ip2_RPT = 0;
  bool ip2_pair = false;                 // paired phi pass possible (tap windows of column pairs)
  int* d_ip2_band = nullptr;
  // staged single right-hand-side FP32 anterpolation into this level
  // (k_anterp2): child theta-row tiles of an2_TI rows (even, so row pairs
  // align), each with the parent rows [lo, hi) it reads ([2][nit], widest
  // an2_BR); an2_PM / an2_TM the widest phi- / theta-transposed stencil; wrap
  // padding of the parent rows an2_PADL left and an2_PADR right; the packed
  // theta taps of each child row (tp | refl << 16) with their weights, used
  // where a row pair reaches a pole
  int an2_TI = 0, an2_nit = 0, an2_BR = 0, an2_PM = 0, an2_TM = 0, an2_PADL = 0, an2_PADR = 0;
  int* d_an2_lo = nullptr;
  int* d_an2_ttp = nullptr;
  float* d_an2_tw = nullptr;
  // pairs of neighbouring child columns / rows (two outputs per thread from one
  // window): window start and dense weights [pairs][2][(PM + 2) or (TM + 3),
  // padded to 4]; a row pair's start is -1 where a row reaches a pole
  int* d_an2_pst2 = nullptr;
  float* d_an2_pwp = nullptr;
  int* d_an2_tq = nullptr;
  float* d_an2_twq = nullptr;
  int ant_PM = 0, ant_TM = 0;             // padded transposed taps per child column / row
  int ant_PMx = 0, ant_TMx = 0;           // real maxima
  int* d_ant_pjp = nullptr;
  double* d_ant_pw64 = nullptr;
  float* d_ant_pw32 = nullptr;
  int* d_ant_ttp = nullptr;
  double* d_ant_tw64 = nullptr;
  float* d_ant_tw32 = nullptr;
  // spectra (allocated for the current R and precision)
  void* d_out = nullptr;                 // active spectra (the last product's precision)
  void* d_in = nullptr;
  size_t spec_bytes = 0;
  void* buf_out[2] = {nullptr, nullptr};   // per precision (SMR_PREC_FP64, SMR_PREC_FP32)
  void* buf_in[2] = {nullptr, nullptr};
  size_t buf_bytes[2] = {0, 0};
};

struct NN {
  int F = 448, H = 0, O = 0, nl = 4;
  int dims[5] = {0, 0, 0, 0, 0};
  long long np = 0;                     // parameter count
  float* p32 = nullptr;                 // master parameters (W_l [in][out] then b_l [out], per layer)
  __nv_bfloat16* w16 = nullptr;         // BF16 copies of the weight matrices (same offsets)
  float *m = nullptr, *v = nullptr, *g = nullptr;
  long long step = 0;
  int cap = 0;                          // rows of the activation buffers
  float* act = nullptr;                 // activations and pre-activations
  float* dact = nullptr;
  double* d_loss = nullptr;
  int* d_slots = nullptr;               // [48][2] neighbour offsets, sorted
};

// one profiled launch: algorithmic bytes / flops and CUDA events around it
struct ProfRec {
  const char* name;
  int level;
  double bytes, flops;
  cudaEvent_t a, b;
};

struct Ctx {
  smr_opts opts;
  std::vector<ProfRec>* prof = nullptr;   // non-null while smr_profile_matvec runs
  std::string err;
  int device = 0;
  std::vector<Shape> shapes;
  bool have_scene = false;
  // scene
  int p = 0, npsi = 0, S = 0, nlev = 0, n_arrays = 1;
  double k = 0, zeta = 1, k_in = 0, zeta_in = 1;
  std::vector<double> centres;          // [p][3]
  std::vector<int> sid;                 // [p]
  std::vector<int> pi, pj;              // lattice indices
  double origin[2] = {0, 0}, z0 = 0;
  std::vector<Level> lev;
  // surface rule (shared by all shapes, scaled by radius)
  int Q = 0;
  std::vector<double> rule_th, rule_ph, rule_w1;  // unit-sphere rule
  double* d_modes = nullptr;            // [S][npsi][Q][4]: psi xyz, div
  double* d_rq = nullptr;               // [S][Q][4]: point xyz, weight
  // patterns [S][npsi][2][K0]
  double2* d_P64 = nullptr;
  float2* d_P32 = nullptr;
  // particles
  int* d_sid = nullptr;
  std::vector<int> arr;                 // [p] array id of each particle
  int* d_arr = nullptr;
  double* d_centres = nullptr;          // [p][3]
  double* d_dshift = nullptr;           // [p][3] r_mu - c_box (finest level)
  int any_dshift = 0;
  // several particles in one finest box: the boxes are the occupied cells,
  // aggregation sums each box's particles and receive reads its box
  int multi = 0;
  std::vector<int> cell_of;              // [p] finest box of each particle
  int* d_cell_of = nullptr;
  int* d_cell_ptr = nullptr;             // [nbox0 + 1] CSR of each box's particles
  int* d_cell_idx = nullptr;             // [p]
  void* pspec[2] = {nullptr, nullptr};   // per-particle level-0 spectra (FP64, FP32)
  // near SpMV: CSR by particle, block ids; blocks stored transposed [nb][2n][2n]
  std::vector<int> nr_ptr, nr_col, nr_blk;
  int* d_nr_ptr = nullptr;
  int* d_nr_col = nullptr;
  int* d_nr_blk = nullptr;
  int nblk = 0;
  std::vector<int> blk_sm, blk_sn, blk_dx, blk_dy;  // key of each block
  std::vector<double> blk_off;            // [nblk][3] r_mu - r_nu of each block
  double2* d_B64 = nullptr;
  float2* d_B32 = nullptr;
  // preconditioner: inverse self blocks, transposed [S][2n][2n]
  bool pinv_ok = true;                  // every self block was invertible
  double2* d_Pinv64 = nullptr;
  float2* d_Pinv32 = nullptr;
  int* d_pc_ptr = nullptr;              // identity CSR for the block kernel
  int* d_pc_col = nullptr;
  int* d_pc_blk = nullptr;
  // particles grouped by shape in tiles of at most 16 (aggregation / receive)
  int ntile = 0;
  int* d_tile_shape = nullptr;
  int* d_tile_start = nullptr;
  int* d_tile_count = nullptr;
  int* d_perm = nullptr;                // particles sorted by shape
  NN nn;
  // captured products: (x, y, R, precision) -> executable graph
  struct GraphEntry {
    const void* x;
    void* y;
    int R, prec;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t capture_stream = nullptr;
  // work buffers
  void* d_G = nullptr;                  // separable-pass intermediate (active precision)
  size_t G_bytes = 0;
  void* G_buf[2] = {nullptr, nullptr};
  size_t G_size[2] = {0, 0};
  int buf_R[2] = {0, 0};
  int spec_R = 0, spec_prec = -1;
  double2* d_tmp = nullptr;             // [N][R] scratch for split products
  size_t tmp_elems = 0;
  // solver scratch
  void* d_sol = nullptr;
  size_t sol_bytes = 0;
  double* d_red = nullptr;              // reduction partials
  size_t red_bytes = 0;
  double* h_red = nullptr;              // pinned host mirror
  // tensor-core receive and aggregation (FP32 product, one right-hand side)
  bool tc_enable = true, tc_ready = false;
  int tc_nK = 0, tc_ntile = 0;
  float* d_tc_rec = nullptr;              // [S][nK][hi | lo][128][32] swizzled coefficient images
  int* d_tc_perm = nullptr;
  int* d_tc_shape = nullptr;
  int* d_tc_start = nullptr;
  int* d_tc_count = nullptr;
  int* d_tc_err = nullptr;                // set when a pipeline wait runs out
  uint32_t tc_spin = 1u << 24;            // polling limit of the pipeline waits (smr_set_wait_limit)
  bool tc_agg_ready = false;
  int tc_nMT = 0, tc_nKc = 0;
  float* d_tc_agg = nullptr;              // [S][M tiles][K chunks][hi | lo][128][32] aggregation images
  // tensor cores for aggregation / receive chosen by smr_autotune (-1: not tuned)
  int tune_tc_agg = -1, tune_tc_rec = -1, tune_tc_near = -1;
  bool lv2_enable = true;                 // staged level kernels for the FP32 product (smr_set_level_kernels)
  // near product on the tensor cores: block images, and per lattice offset
  // (phase; self blocks first) tiles of up to 128 pairs sharing a block
  bool tcn_ready = false;
  int tcn_nK = 0;
  std::vector<int> tcn_phase;             // [n phases + 1] tile ranges
  std::vector<double> tcn_bytes, tcn_flops;   // algorithmic bytes and flops per phase
  float* d_tcn_img = nullptr;             // [nblk][nK][hi | lo][128][32] swizzled block images
  int* d_tcn_blk = nullptr;               // per tile: block
  int* d_tcn_start = nullptr;
  int* d_tcn_count = nullptr;
  int* d_tcn_nu = nullptr;                // per pair: source particle (x row)
  int* d_tcn_mu = nullptr;                // per pair: partial row, phase * p + target particle
  unsigned short* d_tcn_mask = nullptr;   // per particle: phases in which it has a pair
  float* d_tcn_part = nullptr;            // [phase][p][4 n_psi] FP32 partial products
  float2* d_x32 = nullptr;                // x in FP32 for the gathers
  const double2* x32_of = nullptr;        // which x d_x32 holds (set by prep_x32)
  // column buffers of split products ([R][N] in, [R][N] out)
  bool split_cols = true;
  double2* d_split = nullptr;
  size_t split_elems = 0;
  size_t tcn_part_bytes = 0;
  // Column lanes of split products: the columns are dealt round-robin to
  // n_lanes lanes, each with its own FP32 work buffers and stream, so that
  // the small upper-level launches of several columns overlap.  Lane 0 is
  // the context's own buffers and the caller's stream (copied, not owned);
  // lanes 1.. own theirs.
  struct Lane {
    std::vector<void*> out, in;           // per level FP32 spectra
    void* G = nullptr;
    float2* x32 = nullptr;
    float* tcn_part = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;             // end of the lane's columns
  };
  std::vector<Lane> lanes;
  // Overlapped product (smr_set_overlap): per lane a side stream for the
  // translations, one for the near product, and the events that order them
  struct Side {
    cudaStream_t tr = nullptr, nr = nullptr;
    cudaEvent_t ex = nullptr, enear = nullptr;
    std::vector<cudaEvent_t> eout, etr;   // per level: outgoing spectra ready, translation done
  };
  std::vector<Side> side;
  bool overlap = true;
  int cur_side = 0;                       // the side set far_impl uses
  cudaEvent_t near_ev = nullptr;          // the receive waits for it when set
  int n_lanes = 4;                        // columns in flight (smr_set_column_lanes, smr_autotune)
  cudaEvent_t lane_fork = nullptr;
  // cluster block-Jacobi preconditioner (k_cluster.cu): members [ncl][4]
  // (-1 for an absent one), inverses [ncl][4m][4m] transposed, m = 2 n_psi
  bool cl_ready = false;
  int ncl = 0;
  int* d_cl_mem = nullptr;
  double2* d_cl_inv64 = nullptr;
  float2* d_cl_inv32 = nullptr;
  // polynomial preconditioner (smr_solve_opts.poly_degree): roots in Leja
  // order for the running solve, four [N] work vectors, products it made
  std::vector<std::complex<double>> poly_roots;
  bool poly_busy = false;
  int poly_mv = 0;
  double2* d_polyw = nullptr;
  size_t polyw_elems = 0;
  // near-field sweeps preconditioner: three [N][R] work vectors, sweep count
  double2* d_pcw = nullptr;
  size_t pcw_elems = 0;
  int pc_sweeps = 1;
  // learned local-coupling preconditioner: diagonal D [N] (one right-hand side)
  double2* d_lpc = nullptr;
  bool lpc_ready = false;
};

// ------------------------------------------------------------------ helpers
#define SMR_CUDA(ctx, call)                                                        \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return SMR_E_CUDA;                                                           \
    }                                                                              \
  } while (0)

#define SMR_LAUNCH(ctx)                                                            \
  do {                                                                             \
    cudaError_t e_ = cudaGetLastError();                                           \
    if (e_ != cudaSuccess) {                                                       \
      (ctx)->err = std::string("kernel launch: ") + cudaGetErrorString(e_);        \
      return SMR_E_CUDA;                                                           \
    }                                                                              \
  } while (0)

template <typename T>
int upload(Ctx* c, T** dst, const std::vector<T>& src) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (src.empty()) return SMR_OK;
  SMR_CUDA(c, cudaMalloc((void**)dst, src.size() * sizeof(T)));
  SMR_CUDA(c, cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SMR_OK;
}

inline void pbeg(Ctx* c, cudaStream_t st, const char* name, int level, double bytes, double flops) {
  if (!c->prof) return;
  ProfRec r{name, level, bytes, flops, nullptr, nullptr};
  cudaEventCreate(&r.a);
  cudaEventCreate(&r.b);
  cudaEventRecord(r.a, st);
  c->prof->push_back(r);
}
inline void pend(Ctx* c, cudaStream_t st) {
  if (c->prof) cudaEventRecord(c->prof->back().b, st);
}

// ------------------------------------------------------------------ setup (k_setup.cu)
int build_modes(Ctx* c);          // d_modes, d_rq (host evaluation, upload)
int build_patterns(Ctx* c);       // d_P64 / d_P32 on the GPU (FP64)
int build_translations(Ctx* c);   // per level d_T64 / d_T32 on the GPU (FP64)
int build_near(Ctx* c);           // d_B64 / d_B32 on the GPU (FP64) + self blocks
int launch_rhs(Ctx* c, int R, const double* d_khat, const double2* d_pol, double2* b,
               cudaStream_t st);
// R = 1 right-hand side with incidence number arr[mu] for particle mu
// (host khat/pol hold one plane wave per array)
int launch_rhs_arrays(Ctx* c, const double* d_khat, const double2* d_pol, double2* b, cudaStream_t st);
int launch_rhs_scratch(Ctx* c, int R, const double* d_khat, const double2* d_pol, double2* Sv,
                       double2* b, cudaStream_t st);
int launch_far_field(Ctx* c, int R, const double2* x, int nd, const double* d_dirs,
                     double2* F, cudaStream_t st);
int launch_cross_sections(Ctx* c, int R, const double2* x, int n_sca, const double* d_dirs,
                          const double* d_w, const double2* d_pol, double* d_cs, cudaStream_t st);
int launch_near_field(Ctx* c, int R, const double2* x, int npt, const double* d_pts,
                      double2* EH, cudaStream_t st);

// ------------------------------------------------------------------ learned initial guess (k_learned.cu)
int nn_init(Ctx* c, int width, unsigned long long seed);
void nn_free(Ctx* c);
int nn_features(Ctx* c, const double* d_khat, const double* d_pol, float* feat, cudaStream_t st);
int nn_targets(Ctx* c, const double* d_khat, const double2* x, double scale, float* tgt, cudaStream_t st);
int nn_forward_backward(Ctx* c, int n, const float* feat, const int* idx, const float* tgt, bool backward,
                        double* loss_host, cudaStream_t st);
int nn_adam(Ctx* c, float lr, cudaStream_t st);
int nn_predict(Ctx* c, const double* d_khat, const double* d_pol, double scale, double2* x0, cudaStream_t st);
int nn_precond(Ctx* c, const double* d_khat, const double* d_pol, double scale, const double2* b, cudaStream_t st);
int lpc_apply(Ctx* c, double2* z, cudaStream_t st);

// ------------------------------------------------------------------ hot path (k_mlfma.cu)
int ensure_spectra(Ctx* c, int R, int prec);
int run_near(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st);
int run_far(Ctx* c, int R, int prec, const double2* x, double2* y, bool accumulate,
            cudaStream_t st);
int run_precond(Ctx* c, int R, int prec, const double2* r, double2* z, cudaStream_t st);
// y = Z x through a CUDA graph captured on first use for (x, y, R, prec)
int run_matvec_graph(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st);
// y = Z x (near + far); FP32 with R > 1 runs column by column (split products)
int run_product(Ctx* c, int R, int prec, const double2* x, double2* y, cudaStream_t st);
void free_graphs(Ctx* c);
// meshed shapes (mesh.cu)
int mesh_static_modes(Ctx* c, int nv, const double* verts, int nt, const int* tris, int n_perp, int n_par,
                      MeshModes& out);
int mesh_self_block(Ctx* c, const Shape& sh, std::vector<cd>& Z);
// cluster block-Jacobi preconditioner (k_cluster.cu)
bool cluster_ok(const Ctx* c);
int build_clusters(Ctx* c);
int run_cluster(Ctx* c, int R, int prec, const double2* r, double2* z, cudaStream_t st);
void free_clusters(Ctx* c);
// column lanes of split FP32 products (buffers allocated outside graph capture)
int ensure_lanes(Ctx* c, int nl);
void free_lanes(Ctx* c);
int ensure_side(Ctx* c, int n);
void free_side(Ctx* c);
// tensor-core receive and aggregation (k_tc.cu)
int build_tc(Ctx* c);
bool tc_receive_ok(const Ctx* c, int R);
int run_receive_tc(Ctx* c, const float2* in0, double2* y, bool accumulate, cudaStream_t st);
bool tc_aggregate_ok(const Ctx* c, int R);
int build_near_tc(Ctx* c);
bool tc_near_ok(const Ctx* c, int R);
int run_near_tc(Ctx* c, double2* y, cudaStream_t st);
int prep_x32(Ctx* c, int R, int prec, const double2* x, cudaStream_t st);
int run_aggregate_tc(Ctx* c, const double2* x, const float2* x32, float2* out0, cudaStream_t st);
int tc_check(Ctx* c);
// staged FP32 level kernels (k_levels.cu)
bool interp2_ok(const Ctx* c, int s);
int run_interp2(Ctx* c, int s, cudaStream_t st);
bool interp2_pair_ok(const Ctx* c, int s);
bool anterp2_ok(const Ctx* c, int s);
int run_anterp2(Ctx* c, int s, cudaStream_t st);

// ------------------------------------------------------------------ linear algebra (k_linalg.cu)
// h[j*R + r] = sum_i conj(V_j[i][r]) w[i][r] for j < J (V_j = V + j*ldv), FP64.
int multidot(Ctx* c, int J, long long n, int R, const double2* V, long long ldv,
             const double2* w, double2* h_host, cudaStream_t st);
// w[i][r] -= sum_j V_j[i][r] h[j][r]   (h on the device, [J][R])
int multi_axpy(Ctx* c, int J, long long n, int R, const double2* V, long long ldv,
               const double2* d_h, double2* w, double sign, cudaStream_t st);
// norms[r] = ||v[:, r]||_2
int col_norms(Ctx* c, long long n, int R, const double2* v, double* norms_host, cudaStream_t st);
// y[i][r] = a[r] * x[i][r] + b[r] * y[i][r]  (a, b complex per column, device)
int col_axpby(long long n, int R, const double2* d_a, const double2* x, const double2* d_b,
              double2* y, cudaStream_t st);

int solve(Ctx* c, int R, const double2* b, double2* x, const smr_solve_opts* o,
          smr_solve_stats* stats, cudaStream_t st);

}  // namespace smr

// The C ABI wrapper around a context (defined in api.cu).
struct smr_ctx {
  smr::Ctx c;
};
