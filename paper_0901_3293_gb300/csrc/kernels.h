// Host-side entry points of the kernels (internal to liblcbp).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/lcbp.h"
#include "common.cuh"

namespace lcbp {

// Device pointers of one step.  `reps` points to a device array of
// Replica<real>; the field pointers are the bases of the concatenated arrays.
struct StepArgs {
  const void* reps;
  const Tile* tiles;
  int ntiles;
  TileShape ts;
  int flow_on;
  int coupling;  // 0 Jacobi, 1 Gauss-Seidel
  int walls;     // some replica has solid walls in z (selects the bounce-back LB build)
  int div;       // some replica has L2 != K (selects the build with the div Q term of H)
  void* q;       // 5 comps, updated in place
  void* qs;      // 5 comps scratch (Heun predictor)
  void* h;       // 5 comps scratch
  void* sigma;   // 5 comps scratch
  void* tau;     // 3 comps scratch
  void* b;       // 3 comps scratch
  const void* bext;  // 3 comps or nullptr
  void* f;       // 15 comps, step n
  void* fnew;    // 15 comps, step n+1
  void* rhou;    // 4 comps [rho - 1, ux, uy, uz], step n
  void* rhou_new;
  void* qout;    // Q^{n+1}; nullptr = in place on q
  int max_grid;  // > 0: at most this many (persistent) CTAs walk the tile list
  // optional: events[0] is recorded before the first kernel of the step and
  // events[k + 1] after kernel k (per-kernel timing); nullptr otherwise
  cudaEvent_t* events;
};

// number of kernels launch_step issues for a mode
inline int kernels_per_step(int flow_on, int coupling) { return flow_on ? (coupling ? 5 : 3) : 3; }

template <typename real>
cudaError_t launch_step(const StepArgs& a, cudaStream_t s);
template <typename real>
cudaError_t launch_field(const StepArgs& a, cudaStream_t s);
// Beris-Edwards rate R(Q, u) (u = 0 with flow off) written to a.qs
template <typename real>
cudaError_t launch_rate(const StepArgs& a, cudaStream_t s);

// initial Q (kinds as in lcbp.h); per-replica q0 is in q0s[rep] (device array)
struct InitQArgs {
  int kind;
  double amplitude;
  double noise;
  uint64_t seed;
  int z0;
};
template <typename real>
cudaError_t launch_init_q(const void* reps, const Tile* tiles, int ntiles, TileShape ts, const double* q0s,
                          const double* s_helix, const uint64_t* seeds, InitQArgs a, void* q, cudaStream_t s);

// f = f^eq(rho0, u, sigma) with u from u3 (state type, may be null); then moments
template <typename real>
cudaError_t launch_init_feq(const void* reps, const Tile* tiles, int ntiles, TileShape ts, double rho0,
                            const void* u3, const void* sigma, void* f, cudaStream_t s);
template <typename real>
cudaError_t launch_feq_from_moments(const void* reps, const Tile* tiles, int ntiles, TileShape ts, const void* rhou,
                                    const void* sigma, void* f, cudaStream_t s);
template <typename real>
cudaError_t launch_moments(const void* reps, const Tile* tiles, int ntiles, TileShape ts, const void* f,
                           void* rhou, cudaStream_t s);

// deviation storage <-> full values: dst = src + sign * (kind 0: w_c per
// component c of an [comps][n] field; kind 1: 1)
template <typename real>
cudaError_t launch_shift(const void* src, void* dst, long long n, int comps, int kind, int sign, cudaStream_t s);

// element-wise dtype conversion of n values
cudaError_t launch_convert(const void* src, int src_dtype, void* dst, int dst_dtype, long long n, cudaStream_t s);

// Diagnostics of one lattice (replica), accumulated in FP64 with a fixed
// reduction order: out[0..6] = [F_h, mass, Px, Py, Pz, #sites with
// lambda_max(Q) < threshold, #non-finite sites].  partials holds 512 * 8 doubles.
struct DiagGeom {
  int nx, ny, nz;
  long long n, base;
  double A0, gamma, K, q0;
  int walls;       // solid walls in z: F_h in bond form with the anchored ghost planes
  double qw[5];    // anchored Q (q5 order)
  double c_div;    // (K - L2) / 2: F_h gains -c_div |div Q|^2 per site
};
// padded mirror <-> flat field (state.cu): C components of an nx x ny x nz
// field, site (x, y) at column x + hx and row y + hy of a mirror of nxp x nyp
// whose first 4G components are interleaved by fours ([group][z][Y][X][4])
// and whose others are plain arrays; pack fills every mirror position with
// its periodic image
template <typename real>
cudaError_t launch_pack(const void* flat, void* padded, int C, int G, int nx, int ny, int nz, int hx, int hy,
                        int nxp, int nyp, cudaStream_t s);
template <typename real>
cudaError_t launch_unpack(const void* padded, void* flat, int C, int G, int nx, int ny, int nz, int hx, int hy,
                          int nxp, int nyp, cudaStream_t s);

// whole-field checks (state.cu); scratch: state_check_scratch_bytes() of device memory
size_t state_check_scratch_bytes();
// *out = number of non-finite values among n
template <typename real>
cudaError_t launch_count_nonfinite(const void* v, long long n, void* scratch, unsigned long long* out,
                                   cudaStream_t s);
// *out = max |a - b| over n values (NaN if either holds one)
template <typename real>
cudaError_t launch_max_abs_diff(const void* a, const void* b, long long n, void* scratch, double* out,
                                cudaStream_t s);

// one CTA waits on a barrier nothing arrives on, for at most limit_ns; *flag = 1 if it gave up
cudaError_t launch_wait_probe(uint64_t limit_ns, int* flag, cudaStream_t s);
template <typename real>
cudaError_t launch_diag_one(const DiagGeom& g, const void* q, const void* f, int with_f, double threshold,
                            double* partials, double* out, cudaStream_t s);
constexpr int kDiagPartials = 512 * 8;

// ---------------------------------------------------------------------------
// Fast path (flow on, Jacobi coupling, zm_shape_ok): two z-marching kernels
// with TMA-staged planes.  The host builds the tensor maps: the padded mirrors
// of Q and rho u as 3-D tensors (4-D with the replica outermost for a batch
// class), the scratch below as (4 X, Y, group, z), and the populations as a
// 4-D tensor (x, y, z, component) for L2 prefetches.
//
// Between the two kernels the step's intermediate fields live in a
// periodically padded scratch ("LB-ready" scratch) of 16 values per site in
// four groups of four, interleaved per site ([z][group][Y][X][4], one 16-byte
// vector per site and group):
//   G0 = [C, V_x, V_y, V_z], G1 = [W_xy, W_xz, W_yz, F_x],
//   G2 = [F_y, F_z, Q*_yz, rho - 1], G3 = [Q*_xx, Q*_xy, Q*_xz, Q*_yy],
// over an (nx + 4) x (ny + 2) x nz array in which site (x, y, z) sits at
// (X, Y) = (x + 1, y + 1) and the columns x = -1, nx and rows y = -1, ny hold
// the periodic images.  The second kernel then stages them by TMA with no halo
// patching.  F, V, C and W are the per-site coefficients of the LB
// pre-collision terms (f^eq_i / tau_f + p_i of Sec. 2.2 Eq. feq, coeff, eq4):
// a face direction +-e_a has F_a +- V_a, a corner direction s has
// C + (s . V) / 8 + s_x s_y W_xy + s_x s_z W_xz + s_y s_z W_yz.  A corner
// thus reads G0 and G1 of its source site, and the Q* stencil G3 and G2.
// ---------------------------------------------------------------------------
constexpr int kZmPadX = 4;   // padded scratch: columns added to nx (one left, three right)
constexpr int kZmPQ = 16;    // values per site of the padded scratch (four groups of four)
constexpr int kZmPQG = 4;    // groups

struct ZmGeom {
  int nx, ny, nz, zc;
  long long n;
  int tx, ty;  // tile width and rows: 32 x 8 (FP32) or 32 x 4 (FP64); narrow batch tiles 16 x 16
  int tiles_x, tiles_y, tiles_z;
  int nxp, nyp;    // padded scratch and rho u mirror extents: nx + 4, ny + 2
  long long cp;    // their component stride: nxp * nyp * nz
  int nxm;         // mirror row length: zm_mirror_nx(nx)
  int nyq, nyu;    // mirror rows per plane: ny + 4 (Q), ny + 2 (rho u)
  long long cq, cu;  // mirror component strides: nxm * nyq * nz, nxm * nyu * nz
};

// Padded mirrors of the state (single lattices on the fast path): Q and rho u
// with 32 columns before each row and rows of a whole number of 128-byte
// lines in FP32 (site x at column x + 32, so that a warp's row of 32 sites is
// one aligned line), and two (Q) or one (rho u) rows added on each side; the
// ghost columns and rows next to the lattice hold the periodic images
// (x = -2, -1, nx, nx + 1 for Q, -1 and nx for rho u).  Components are
// interleaved by fours, one 16-byte vector per site: rho u as
// [z][Y][X][rho-1, u_x, u_y, u_z], Q as [z][Y][X][xx, xy, xz, yy] followed by
// the plain array [z][Y][X] of yz.  k_lbq writes Q^{n+1} and rho u^{n+1} there,
// images included, so the next step stages them with no patching.
constexpr int kZmMirX = 32;  // columns before x = 0 in a mirror row
// Batch classes of FP32 replicas whose width leaves a last 32-column tile at
// most half full (nx % 32 in 1..16, e.g. 48) take tiles of 16 columns by 16
// rows instead: the same 256 sites and threads, no idle lanes.
constexpr int kZmNarrowX = 16;
inline int zm_batch_tile_x(int nx, bool fp32) { return fp32 && nx % 32 != 0 && nx % 32 <= 16 ? kZmNarrowX : 32; }
inline int zm_mirror_nx(int nx) { return (nx + 31) / 32 * 32 + 2 * kZmMirX; }  // mirror row length
inline long long zm_qmirror_elems(int nx, int ny, int nz) { return 5LL * zm_mirror_nx(nx) * (ny + 4) * nz; }
inline long long zm_umirror_elems(int nx, int ny, int nz) { return 4LL * zm_mirror_nx(nx) * (ny + 2) * nz; }

// Shapes the fast kernels serve: rows of whole 16-byte groups (nx % 4 == 0 for
// the TMA boxes) and element offsets within one lattice that fit in 32 bits
// (the kernels index with int; the largest offsets are those of the 15
// populations, the 16 scratch values and the 5 components of the Q mirror).
inline bool zm_shape_ok(int nx, int ny, int nz) {
  const long long n = (long long)nx * ny * nz, cp = (long long)(nx + kZmPadX) * (ny + 2) * nz;
  const long long cq = (long long)zm_mirror_nx(nx) * (ny + 4) * nz, lim = 2147483647LL;
  return nx % 4 == 0 && 15 * n < lim && kZmPQ * cp < lim && 5 * cq < lim;
}

struct ZmArgs {
  int nx, ny, nz, zc;  // zc: planes per CTA of k_lbq
  int zc_q;           // planes per CTA of k_qside (0: as zc)
  int spt;            // sites per thread of k_lbq, 1 or 2 (2 only where zm_spt_max allows)
  int spt_q;          // sites per thread of k_qside (0: as spt)
  const void* model;  // host copy of Model<real>
  // the Q mirror as [xx xy xz yy] vectors (tm_q) and yz (tm_q1), box rows
  // TY + 4; the rho u mirror (tm_u, 4-vectors; tm_u3 the same for k_lbq); the
  // padded scratch (16 values per site)
  const CUtensorMap *tm_q, *tm_q1, *tm_u, *tm_pq, *tm_u3;
  // f^n for L2 prefetches of the pulled populations: the tile's rows with all
  // 15 components (tm_f), and the halo rows' inward-moving populations in
  // boxes of one (tm_f1) or two (tm_f2) components
  const CUtensorMap *tm_f, *tm_f1, *tm_f2;
  // the Q mirror in boxes of one tile (32 x TY sites, no halo), for k_lbq's L2
  // prefetches of Q^n: it reads Q^n at its own sites only
  const CUtensorMap *tm_qpf, *tm_q1pf;
  void *q, *qout, *pq;  // qout: nullptr = update Q in place; pq: padded scratch
  const void* bext;
  void *f, *fnew, *rhou, *rhou_new;
  int* err;              // set to 1 if a bounded barrier wait timed out
  cudaEvent_t* events;   // optional: 3 events around the two kernels
  const double* q_wall;  // walls in z with this anchored Q (5 values), or nullptr: periodic
};

// elements of the padded scratch of one nx x ny x nz lattice
inline long long zm_pq_elems(int nx, int ny, int nz) {
  return (long long)kZmPQ * (nx + kZmPadX) * (ny + 2) * nz;
}

// box widths of 32-wide tiles (single lattices; batch classes derive theirs from the tile width)
constexpr int kZmBoxX = 40;   // sites per TMA box row of the flat fields and of the Q mirror (x0 - 4 ..)
constexpr int kZmBoxXP = 34;  // sites per TMA box row of the padded scratch (x0 - 1 .. x0 + 32)
constexpr int kZmBoxXU = 34;  // sites per TMA box row of the rho u mirror (x0 - 1 .. x0 + 32)

// Fast path over a batch: replicas of equal dims form a class whose fields are
// stored back to back, so that each field of a class is one 5-D tensor
// (x, y, z, component, replica).  Classes own consecutive CTA ranges of one
// launch per kernel.
constexpr int kZmMaxClasses = 4;
struct ZmClass {
  ZmGeom G;
  int cta0;          // first CTA of the class
  int ctas_per_rep;  // tiles_x * tiles_y * tiles_z
  int rep0;          // first entry of the class in the replica order table
  int count;         // replicas in the class
  long long pq0;     // first element of the class's padded scratch (replica j at pq0 + j * 16 * cp)
  long long qm0;     // first element of the class's Q mirrors (replica j at qm0 + j * 5 * cq)
  long long um0;     // first element of the class's rho u mirrors (replica j at um0 + j * 4 * cu)
};
struct ZmBatch {
  int nclass;
  int total_ctas;
  ZmClass c[kZmMaxClasses];
};
// Per class, with the replica as the outermost coordinate: the Q mirrors'
// [xx xy xz yy] vectors (q) and yz arrays (q1), the rho u mirrors (u; u3 the
// same for k_lbq) and the padded scratch (pq, 5-D).  Boxes fit the class's
// tile of tx x ty sites: Q tx + 8 sites wide (from x0 - 4) and ty + 4 rows,
// the others tx + 2 wide and ty + 2 rows.  For k_lbq's L2 prefetches only:
// the Q mirrors in tile-sized boxes (qpf, q1pf) and the flat populations as
// 5-D tensors (x, y, z, i, replica), tx + 8 wide, in boxes of the tile's rows
// with all 15 populations (f) or of one halo row with one (f1) or two (f2).
struct ZmBatchMaps {
  CUtensorMap q[kZmMaxClasses], q1[kZmMaxClasses], u[kZmMaxClasses], pq[kZmMaxClasses], u3[kZmMaxClasses],
      f[kZmMaxClasses], qpf[kZmMaxClasses], q1pf[kZmMaxClasses], f1[kZmMaxClasses], f2[kZmMaxClasses];
};
struct ZmBatchArgs {
  ZmBatch B;   // classes and CTA ranges of k_lbq_batch
  ZmBatch Bq;  // the same for k_qside_batch (its own planes per CTA)
  const ZmBatchMaps* maps;  // host copy (rho u maps of the current buffer)
  const void* reps;         // device Replica<real>[R]: base offsets and models
  const int* order;         // device: replica indices, class by class in storage order
  void *q, *qout, *pq;      // Q mirrors of all classes; qout: nullptr = update them in place; pq: padded scratch
  void *f, *fnew;           // the flat populations
  void *rhou, *rhou_new;    // rho u mirrors of all classes (current, next)
  int* err;
  cudaEvent_t* events;      // optional: recorded before, between and after the two kernels
};
template <typename real>
cudaError_t zm_batch_prepare();
template <typename real>
cudaError_t launch_step_zm_batch(const ZmBatchArgs& a, cudaStream_t s);
template <typename real>
int zm_tile_rows();
// polarised texture of a Q field into a device image [ny][nx] (optics.cu)
// d_img: nx * ny image followed by scratch; scratch_floats counts both
template <typename real>
cudaError_t launch_texture(const void* q, int nx, int ny, int nz, const lcbp_optics& o, float* d_img,
                           long long scratch_floats, cudaStream_t s);

template <typename real>
int zm_spt_max();
template <typename real>
int zm_resident(int spt);  // k_lbq CTAs resident per SM
template <typename real>
cudaError_t zm_prepare();
template <typename real>
cudaError_t launch_step_zm(const ZmArgs& a, cudaStream_t s);

}  // namespace lcbp
