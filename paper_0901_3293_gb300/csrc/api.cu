// C ABI of liblcbp: lattice handle, memory, parameters, stepping (CUDA graph
// replay), transfers, diagnostics and checkpoints.  See include/lcbp.h.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lcbp.h"
#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

using namespace lcbp;

namespace lcbp {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LCBP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

TileShape default_tile(int nx, int ny, int nz) {
  TileShape t;
  t.tx = std::min(nx, 32);
  t.ty = std::min(ny, std::max(1, 128 / t.tx));
  t.tz = std::min(nz, std::max(1, 128 / (t.tx * t.ty)));
  return t;
}

long long tile_count(int nx, int ny, int nz, TileShape t) {
  return (long long)((nx + t.tx - 1) / t.tx) * ((ny + t.ty - 1) / t.ty) * ((nz + t.tz - 1) / t.tz);
}

void append_tiles(std::vector<Tile>& out, int rep, int nx, int ny, int nz, TileShape t) {
  for (int z = 0; z < nz; z += t.tz)
    for (int y = 0; y < ny; y += t.ty)
      for (int x = 0; x < nx; x += t.tx) out.push_back(Tile{rep, x, y, z});
}

bool valid_dtype(int d) { return d == LCBP_F32 || d == LCBP_F64; }
size_t dtype_size(int d) { return d == LCBP_F64 ? 8 : 4; }

// Model coefficients in the state type, from double parameters
template <typename real>
Model<real> make_model(const HostParams& p) {
  Model<real> m;
  m.a_bulk = (real)(p.A0 * (1.0 - p.gamma / 3.0));
  m.b_bulk = (real)(p.A0 * p.gamma);
  m.K = (real)p.K;
  m.kq0x2 = (real)(2.0 * p.K * p.q0);
  m.kq0sq4 = (real)(4.0 * p.K * p.q0 * p.q0);
  m.Gamma = (real)p.Gamma;
  m.xi = (real)p.xi;
  m.inv_tau = (real)(1.0 / p.tau_f);
  m.c_div = (real)(p.l2_set ? 0.5 * (p.K - p.L2) : 0.0);
  return m;
}

template <typename real>
void fill_replica(void* dst, int nx, int ny, int nz, long long base, const HostParams& p) {
  Replica<real> r{};
  r.nx = nx;
  r.ny = ny;
  r.nz = nz;
  r.n = (long long)nx * ny * nz;
  r.base = base;
  r.m = make_model<real>(p);
  r.walls = p.walls_z;
  for (int c = 0; c < 5; ++c) r.qw[c] = (real)p.q_wall[c];
  std::memcpy(dst, &r, sizeof(r));
}
template void fill_replica<float>(void*, int, int, int, long long, const HostParams&);
template void fill_replica<double>(void*, int, int, int, long long, const HostParams&);

size_t replica_bytes(int dtype) { return dtype == LCBP_F64 ? sizeof(Replica<double>) : sizeof(Replica<float>); }

double s_eq(double gamma) {
  const double d = 1.0 - 8.0 / (3.0 * gamma);
  return d > 0 ? 0.25 + 0.75 * std::sqrt(d) : 0.0;
}

int check_params(const HostParams& p) {
  const double v[] = {p.A0, p.gamma, p.K, p.q0, p.tau_f, p.xi, p.Gamma};
  for (double x : v)
    if (!std::isfinite(x)) return fail(LCBP_EINVAL, "non-finite parameter");
  if (p.A0 <= 0 || p.gamma <= 0 || p.K < 0) return fail(LCBP_EINVAL, "need A0 > 0, gamma > 0, K >= 0");
  if (p.tau_f <= 0 || p.Gamma < 0) return fail(LCBP_EINVAL, "need tau_f > 0, Gamma >= 0");
  if (p.coupling != LCBP_JACOBI && p.coupling != LCBP_GAUSS_SEIDEL) return fail(LCBP_EINVAL, "bad coupling");
  return LCBP_OK;
}

// Copy `count` values between a caller buffer (host or device, dtype `ud`)
// and a device state array (dtype `sd`), converting through `staging`.
int transfer(void* state, int sd, void* user, int ud, long long count, bool upload, void* staging,
             long long staging_elems, cudaStream_t st) {
  cudaError_t e;
  if (ud == sd) {
    const size_t bytes = (size_t)count * dtype_size(sd);
    e = upload ? cudaMemcpyAsync(state, user, bytes, cudaMemcpyDefault, st)
               : cudaMemcpyAsync(user, state, bytes, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "cudaStreamSynchronize");
  }
  const size_t ues = dtype_size(ud), ses = dtype_size(sd);
  for (long long off = 0; off < count; off += staging_elems) {
    const long long m = std::min(staging_elems, count - off);
    if (upload) {
      e = cudaMemcpyAsync(staging, static_cast<char*>(user) + off * ues, m * ues, cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
      e = launch_convert(staging, ud, static_cast<char*>(state) + off * ses, sd, m, st);
    } else {
      e = launch_convert(static_cast<char*>(state) + off * ses, sd, staging, ud, m, st);
      if (e != cudaSuccess) return cuda_fail(e, "convert");
      e = cudaMemcpyAsync(static_cast<char*>(user) + off * ues, staging, m * ues, cudaMemcpyDefault, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "transfer");
    e = cudaStreamSynchronize(st);  // staging is reused by the next chunk
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  }
  return LCBP_OK;
}


// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda
// link): a tiled map with unit element strides, no swizzle or interleave,
// 128-byte L2 promotion and zero fill.  strides: rank - 1 byte strides.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_tiled(CUtensorMap* tm, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
                  const cuuint32_t* box, int dtype) {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  if (!fn || rank < 1 || rank > 5) return false;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(tm, dtype == LCBP_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base,
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace lcbp

// ---------------------------------------------------------------------------
// lattice handle
// ---------------------------------------------------------------------------
struct lcbp_lattice {
  int nx, ny, nz;
  long long n;
  int dtype;
  size_t es;
  int device;
  HostParams p{};
  cudaStream_t stream;
  bool own_stream;
  char* ws;
  size_t ws_bytes;
  bool own_ws;
  // state and scratch (device)
  void *f[2], *rhou[2], *q, *qs, *h, *sig, *tau, *b, *bext, *staging;
  void* pq;  // the fast kernels' padded scratch (overlays h, sig, tau, b)
  void *qm, *um[2];  // padded mirrors of Q and rho u [0] / [1] (fast path)
  bool flat_ok;      // q and rhou[cur] hold the current state
  bool mirror_ok;    // qm and um[cur] hold the current state
  long long staging_elems;
  void* d_rep;
  Tile* d_tiles;
  int ntiles;
  TileShape ts;
  double *d_q0, *d_shelix;
  uint64_t* d_seed;
  double *d_partials, *d_out;
  double* h_out;  // pinned
  int cur;
  bool f_ready, has_bext;
  cudaGraphExec_t graph;
  bool graph_ok;
  long long step;
  // fast path (z-marching TMA kernels)
  int path_req;   // LCBP_PATH_*
  bool tmaps_ok;  // tensor maps built
  int zc;         // planes per CTA of k_lbq, 0 until tuned
  int zc_q;       // planes per CTA of k_qside, set by the tuner
  int spt;        // sites per thread of k_lbq, set by the tuner
  int spt_q;      // sites per thread of k_qside, set by the tuner
  // Q mirror vectors, rho u mirror [0], [1], padded scratch, (unused), (unused), f [0], f [1], Q mirror yz
  CUtensorMap tm[13];
  int* d_err;
};

namespace {

struct Layout {
  size_t off[19];
  size_t total;
};

constexpr long long kStagingMax = 1ll << 22;  // elements of the conversion buffer

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// offsets of: f0 f1 rhou0 rhou1 q qs h sig tau b bext staging rep tiles q0/shelix/seed partials.
// h, sig, tau and b (the generic kernels' scratch) lie back to back in one
// block, and the fast kernels' padded scratch overlays that block from its
// start: the two kernel sets never run within one step, and no scratch
// outlives a step.
Layout layout(int nx, int ny, int nz, int dtype) {
  const long long n = (long long)nx * ny * nz;
  const size_t es = dtype_size(dtype);
  const TileShape ts = default_tile(nx, ny, nz);
  const long long nt = tile_count(nx, ny, nz, ts);
  const long long comps[6] = {15, 15, 4, 4, 5, 5};
  Layout L{};
  size_t o = 0;
  for (int i = 0; i < 6; ++i) {
    L.off[i] = o;
    o = align256(o + (size_t)(comps[i] * n) * es);
  }
  // (the padded scratch, then a Q-mirror-sized buffer for the tuner's output)
  const long long scr = std::max(16 * n, zm_pq_elems(nx, ny, nz) + zm_qmirror_elems(nx, ny, nz));
  L.off[6] = o;
  L.off[7] = o + (size_t)(5 * n) * es;
  L.off[8] = o + (size_t)(10 * n) * es;
  L.off[9] = o + (size_t)(13 * n) * es;
  o = align256(o + (size_t)scr * es);
  L.off[10] = o;  // external body force
  o = align256(o + (size_t)(3 * n) * es);
  L.off[11] = o;  // staging (doubles)
  o = align256(o + (size_t)std::min(kStagingMax, 15 * n) * 8);
  L.off[12] = o;  // replica table
  o = align256(o + replica_bytes(dtype));
  L.off[13] = o;  // tiles
  o = align256(o + (size_t)nt * sizeof(Tile));
  L.off[14] = o;  // q0, s_helix, seed, error flag
  o = align256(o + 64);
  L.off[15] = o;  // partials + out
  o = align256(o + (kDiagPartials + 8) * 8);
  // padded mirrors of Q and rho u [0], [1] (lattices the fast path can serve)
  const bool fast_shape = zm_shape_ok(nx, ny, nz);
  L.off[16] = o;
  o = align256(o + (fast_shape ? (size_t)zm_qmirror_elems(nx, ny, nz) * es : 0));
  L.off[17] = o;
  o = align256(o + (fast_shape ? (size_t)zm_umirror_elems(nx, ny, nz) * es : 0));
  L.off[18] = o;
  o = align256(o + (fast_shape ? (size_t)zm_umirror_elems(nx, ny, nz) * es : 0));
  L.total = o;
  return L;
}

int check_dims(int nx, int ny, int nz) {
  if (nx < 1 || ny < 1 || nz < 1) return fail(LCBP_EINVAL, "lattice sizes must be >= 1");
  if ((long long)nx * ny * nz > (1ll << 31)) return fail(LCBP_EINVAL, "more than 2^31 sites");
  return LCBP_OK;
}

void drop_graph(lcbp_lattice* h);

int upload_replica(lcbp_lattice* h) {
  drop_graph(h);  // the fast path takes the model coefficients as kernel arguments
  std::vector<char> buf(replica_bytes(h->dtype));
  if (h->dtype == LCBP_F64) fill_replica<double>(buf.data(), h->nx, h->ny, h->nz, 0, h->p);
  else fill_replica<float>(buf.data(), h->nx, h->ny, h->nz, 0, h->p);
  const double aux[2] = {h->p.q0, s_eq(h->p.gamma)};
  cudaError_t e = cudaMemcpyAsync(h->d_rep, buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q0, aux, sizeof(aux), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "upload parameters");
}

int finish_create(lcbp_lattice* h) {
  const Layout L = layout(h->nx, h->ny, h->nz, h->dtype);
  char* w = h->ws;
  h->f[0] = w + L.off[0];
  h->f[1] = w + L.off[1];
  h->rhou[0] = w + L.off[2];
  h->rhou[1] = w + L.off[3];
  h->q = w + L.off[4];
  h->qs = w + L.off[5];
  h->h = w + L.off[6];
  h->sig = w + L.off[7];
  h->tau = w + L.off[8];
  h->b = w + L.off[9];
  h->bext = w + L.off[10];
  h->pq = h->h;
  h->qm = w + L.off[16];
  h->um[0] = w + L.off[17];
  h->um[1] = w + L.off[18];
  h->flat_ok = true;
  h->mirror_ok = false;
  h->staging = w + L.off[11];
  h->staging_elems = std::min(kStagingMax, 15 * h->n);
  h->d_rep = w + L.off[12];
  h->d_tiles = reinterpret_cast<Tile*>(w + L.off[13]);
  h->d_q0 = reinterpret_cast<double*>(w + L.off[14]);
  h->d_shelix = h->d_q0 + 1;
  h->d_seed = reinterpret_cast<uint64_t*>(h->d_q0 + 2);
  h->d_err = reinterpret_cast<int*>(h->d_q0 + 3);
  h->d_partials = reinterpret_cast<double*>(w + L.off[15]);
  h->d_out = h->d_partials + kDiagPartials;
  h->ts = default_tile(h->nx, h->ny, h->nz);
  std::vector<Tile> tiles;
  append_tiles(tiles, 0, h->nx, h->ny, h->nz, h->ts);
  h->ntiles = (int)tiles.size();
  cudaError_t e = cudaMemsetAsync(h->ws, 0, L.off[11], h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(w + L.off[14], 0, 64, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_out, 8 * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "lattice set-up");
  return upload_replica(h);
}

HostParams default_params() {
  HostParams p{};
  p.A0 = 0.01;
  p.gamma = 3.1;
  p.K = 0.01;
  p.q0 = 2.0 * M_PI / 16.0;
  p.tau_f = 2.0;
  p.xi = 0.7;
  p.Gamma = 0.3;
  p.flow_on = 1;
  p.coupling = LCBP_JACOBI;
  p.rho0 = 1.0;
  return p;
}

lcbp_lattice* new_handle(int nx, int ny, int nz, int dtype) {
  auto* h = new lcbp_lattice();
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->n = (long long)nx * ny * nz;
  h->dtype = dtype;
  h->es = dtype_size(dtype);
  h->p = default_params();
  cudaGetDevice(&h->device);
  return h;
}

// ---- fast path: tensor maps, eligibility, autotuned z-chunk -------------------
// field [comps][nz][ny][nx] as a 4-D tensor, box = 40 x rows x 1 x box_comps
bool make_field_tmap(CUtensorMap* tm, void* base, int comps, int nx, int ny, int nz, int rows, int box_comps,
                     int dtype) {
  const cuuint64_t es = dtype_size(dtype);
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)comps};
  const cuuint64_t strides[3] = {nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
  const cuuint32_t box[4] = {(cuuint32_t)kZmBoxX, (cuuint32_t)rows, 1, (cuuint32_t)box_comps};
  return encode_tiled(tm, base, 4, dims, strides, box, dtype);
}

// one plane-interleaved mirror array [nz][nym][w] (w elements per row) as a
// 3-D tensor, box = inner x rows x 1
bool make_mirror_tmap(CUtensorMap* tm, void* base, int w, int nym, int nz, int inner, int rows, int dtype) {
  const cuuint64_t es = dtype_size(dtype);
  const cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)nym, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)w * es, (cuuint64_t)w * nym * es};
  const cuuint32_t box[3] = {(cuuint32_t)inner, (cuuint32_t)rows, 1};
  return encode_tiled(tm, base, 3, dims, strides, box, dtype);
}

// the LB-ready scratch [z][group][nyp][nxp][4] as a 4-D tensor (4 nxp, nyp,
// group, z), box = 4 * 34 x rows x 4 groups x 1
bool make_scratch_tmap(CUtensorMap* tm, void* base, int nxp, int nyp, int nz, int rows, int dtype) {
  const cuuint64_t es = dtype_size(dtype), X = 4 * (cuuint64_t)nxp;
  const cuuint64_t dims[4] = {X, (cuuint64_t)nyp, (cuuint64_t)kZmPQG, (cuuint64_t)nz};
  const cuuint64_t strides[3] = {X * es, X * nyp * es, (cuuint64_t)kZmPQ * nxp * nyp * es};
  const cuuint32_t box[4] = {(cuuint32_t)(4 * kZmBoxXP), (cuuint32_t)rows, (cuuint32_t)kZmPQG, 1};
  return encode_tiled(tm, base, 4, dims, strides, box, dtype);
}

bool fast_shape_ok(const lcbp_lattice* h) { return zm_shape_ok(h->nx, h->ny, h->nz); }

bool use_fast(lcbp_lattice* h) {
  if (h->path_req == LCBP_PATH_GENERIC || !h->p.flow_on || h->p.coupling != LCBP_JACOBI || !fast_shape_ok(h) ||
      (h->p.l2_set && h->p.L2 != h->p.K))
    return false;
  if (!h->tmaps_ok) {
    static std::once_flag prep32, prep64;
    if (h->dtype == LCBP_F64) std::call_once(prep64, [] { zm_prepare<double>(); });
    else std::call_once(prep32, [] { zm_prepare<float>(); });
    const int ty = h->dtype == LCBP_F64 ? zm_tile_rows<double>() : zm_tile_rows<float>();
    // Q and rho u from their padded mirrors (40- and 34-site boxes; Q as its
    // [xx xy xz yy] vectors and its yz array), and the LB-ready scratch
    // (34-site boxes)
    const int nxm = zm_mirror_nx(h->nx), nyq = h->ny + 4, nyu = h->ny + 2;
    const long long cq = (long long)nxm * nyq * h->nz;
    bool ok = make_mirror_tmap(&h->tm[0], h->qm, 4 * nxm, nyq, h->nz, 4 * kZmBoxX, ty + 4, h->dtype) &&
              make_mirror_tmap(&h->tm[8], static_cast<char*>(h->qm) + 4 * cq * h->es, nxm, nyq, h->nz, kZmBoxX,
                               ty + 4, h->dtype) &&
              // the same in tile-sized boxes (k_lbq's prefetches of Q^n at its own sites)
              make_mirror_tmap(&h->tm[4], h->qm, 4 * nxm, nyq, h->nz, 4 * 32, ty, h->dtype) &&
              make_mirror_tmap(&h->tm[5], static_cast<char*>(h->qm) + 4 * cq * h->es, nxm, nyq, h->nz, 32, ty,
                               h->dtype);
    for (int k = 0; k < 2; ++k)
      ok = ok && make_mirror_tmap(&h->tm[1 + k], h->um[k], 4 * nxm, nyu, h->nz, 4 * kZmBoxXU, ty + 2, h->dtype);
    const int nxp = h->nx + kZmPadX;
    ok = ok && make_scratch_tmap(&h->tm[3], h->pq, nxp, nyu, h->nz, ty + 2, h->dtype);
    for (int k = 0; k < 2; ++k) {  // the populations (L2 prefetches only): the tile's rows, then halo-row boxes
      ok = ok && make_field_tmap(&h->tm[6 + k], h->f[k], NV, h->nx, h->ny, h->nz, ty, NV, h->dtype);
      ok = ok && make_field_tmap(&h->tm[9 + k], h->f[k], NV, h->nx, h->ny, h->nz, 1, 1, h->dtype);
      ok = ok && make_field_tmap(&h->tm[11 + k], h->f[k], NV, h->nx, h->ny, h->nz, 1, 2, h->dtype);
    }
    if (!ok) {
      h->path_req = LCBP_PATH_GENERIC;  // tensor maps unavailable: stay on the generic kernels
      return false;
    }
    h->tmaps_ok = true;
  }
  return true;
}

ZmArgs zm_args(lcbp_lattice* h, const void* model) {
  ZmArgs a{};
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.zc = h->zc > 0 ? h->zc : std::min(h->nz, 32);
  a.zc_q = h->zc_q > 0 ? h->zc_q : a.zc;
  a.spt = h->spt > 0 ? h->spt : 1;
  a.spt_q = h->spt_q > 0 ? h->spt_q : a.spt;
  a.model = model;
  a.tm_q = &h->tm[0];
  a.tm_q1 = &h->tm[8];
  a.tm_u = &h->tm[1 + h->cur];
  a.tm_pq = &h->tm[3];
  a.tm_u3 = &h->tm[1 + h->cur];
  a.tm_f = &h->tm[6 + h->cur];
  a.tm_f1 = &h->tm[9 + h->cur];
  a.tm_f2 = &h->tm[11 + h->cur];
  a.tm_qpf = &h->tm[4];
  a.tm_q1pf = &h->tm[5];
  a.q = h->qm;
  a.qout = nullptr;
  a.pq = h->pq;
  a.bext = h->has_bext ? h->bext : nullptr;
  a.f = h->f[h->cur];
  a.fnew = h->f[h->cur ^ 1];
  a.rhou = h->um[h->cur];
  a.rhou_new = h->um[h->cur ^ 1];
  a.err = h->d_err;
  a.events = nullptr;
  a.q_wall = h->p.walls_z ? h->p.q_wall : nullptr;
  return a;
}

struct ModelBuf {
  alignas(16) char bytes[sizeof(Model<double>)];
};

ModelBuf host_model(const lcbp_lattice* h) {
  ModelBuf mb{};
  if (h->dtype == LCBP_F64) {
    const Model<double> m = make_model<double>(h->p);
    std::memcpy(mb.bytes, &m, sizeof(m));
  } else {
    const Model<float> m = make_model<float>(h->p);
    std::memcpy(mb.bytes, &m, sizeof(m));
  }
  return mb;
}

cudaError_t launch_zm(lcbp_lattice* h, const ZmArgs& a) {
  return h->dtype == LCBP_F64 ? launch_step_zm<double>(a, h->stream) : launch_step_zm<float>(a, h->stream);
}

// planes per CTA and sites per thread of each fast kernel, chosen by timing
// each candidate once per lattice shape and dtype (each kernel by its own
// events, so each takes its own best); the runs write only scratch buffers
// (Q^{n+1} to a Q-mirror-sized scratch), so the state is untouched.  Results
// are kept per process and, if the environment variable LCBP_AUTOTUNE_CACHE
// names a file, in that file ("nx ny nz dtype zc spt [zc_q]" per line, dtype +
// 100 with walls, zc / zc_q = planes per CTA of k_lbq / k_qside (zc_q as zc
// if absent), spt = sites per thread of k_lbq + 10 x those of k_qside).
struct Tuning {
  int zc, spt, zc_q;
};
std::mutex g_tune_mu;
std::map<std::string, Tuning> g_tune;
bool g_tune_loaded = false;

// "nx ny nz dtype", with 100 added to dtype for a lattice with walls
std::string tune_key(const lcbp_lattice* h) {
  char k[64];
  snprintf(k, sizeof(k), "%d %d %d %d", h->nx, h->ny, h->nz, h->dtype + (h->p.walls_z ? 100 : 0));
  return k;
}

// Planes-per-CTA candidates: the powers of two, and the values that make the
// grid (column tiles x z-chunks) fill a whole number of waves of resident CTAs
// or fall just short of one, for 1 to 48 waves.  All lie in [4, 64] (or are nz).
std::vector<int> zc_candidates(const lcbp_lattice* h, int spt) {
  std::vector<int> c;
  for (int zc : {4, 8, 16, 32, 64})
    if (zc <= h->nz) c.push_back(zc);
  if (h->nz < 64) c.push_back(h->nz);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ty = h->dtype == LCBP_F64 ? zm_tile_rows<double>() : zm_tile_rows<float>();
  const long long tiles_xy = (long long)((h->nx + 31) / 32) * ((h->ny + ty - 1) / ty);
  const long long resident = (long long)sms * (h->dtype == LCBP_F64 ? zm_resident<double>(spt) : zm_resident<float>(spt));
  for (int w = 1; w <= 48; ++w) {
    const long long want = w * resident;
    for (long long chunks : {want / tiles_xy, (want + tiles_xy - 1) / tiles_xy}) {
      if (chunks < 1) continue;
      const long long zc = (h->nz + chunks - 1) / chunks;
      if (zc >= 4 && zc <= 64) c.push_back((int)zc);
    }
  }
  std::sort(c.begin(), c.end());
  c.erase(std::unique(c.begin(), c.end()), c.end());
  return c;
}

int tune_zc(lcbp_lattice* h) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const char* path = std::getenv("LCBP_AUTOTUNE_CACHE");
  const int spt_max = h->dtype == LCBP_F64 ? zm_spt_max<double>() : zm_spt_max<float>();
  // a pinned sites-per-thread choice tunes only the planes per CTA, uncached
  const bool pinned = h->path_req == LCBP_PATH_FAST1 || h->path_req == LCBP_PATH_FAST2;
  // (walls: one site per thread only)
  const int spt_lo = h->path_req == LCBP_PATH_FAST2 && !h->p.walls_z ? 2 : 1;
  const int spt_hi = h->path_req == LCBP_PATH_FAST1 || h->p.walls_z ? 1 : spt_max;
  if (path && !g_tune_loaded) {
    g_tune_loaded = true;
    if (FILE* fp = std::fopen(path, "r")) {
      char line[256];
      while (std::fgets(line, sizeof(line), fp)) {
        int a, b, c, d, z, sp, zq = 0;
        const int got = std::sscanf(line, "%d %d %d %d %d %d %d", &a, &b, &c, &d, &z, &sp, &zq);
        if (got < 6) continue;
        if (got == 6) zq = z;
        char k[64];
        snprintf(k, sizeof(k), "%d %d %d %d", a, b, c, d);
        if (z >= 1 && zq >= 1 && sp % 10 >= 1 && sp % 10 <= 2 && sp / 10 >= 1 && sp / 10 <= 2)
          g_tune[k] = {z, sp, zq};
      }
      std::fclose(fp);
    }
  }
  const std::string key = tune_key(h);
  auto it = g_tune.find(key);
  if (!pinned && it != g_tune.end() && it->second.spt % 10 <= spt_max && it->second.spt / 10 <= spt_max) {
    h->zc = it->second.zc;
    h->zc_q = it->second.zc_q;
    h->spt = it->second.spt % 10;
    h->spt_q = it->second.spt / 10;
    return LCBP_OK;
  }
  const ModelBuf mb = host_model(h);
  cudaEvent_t ev[3];
  for (int i = 0; i < 3; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) return fail(LCBP_ECUDA, "event create");
  auto destroy = [&]() {
    for (int i = 0; i < 3; ++i) cudaEventDestroy(ev[i]);
  };
  // each kernel keeps its own best: k_lbq over (spt, zc), k_qside over (spt_q, zc)
  float best_l = 1e30f, best_q = 1e30f;
  int best_zc = std::min(h->nz, 32), best_zq = best_zc, best_spt = spt_lo, best_sq = spt_lo;
  for (int spt = spt_lo; spt <= spt_hi; ++spt) {
    for (int sq = spt_lo; sq <= spt_hi; ++sq) {
      for (int zc : zc_candidates(h, spt)) {
        ZmArgs a = zm_args(h, mb.bytes);
        a.zc = a.zc_q = zc;
        a.spt = spt;
        a.spt_q = sq;
        a.events = ev;  // before k_qside, between the kernels, after k_lbq
        // Q^{n+1} to the Q-mirror-sized buffer after the padded scratch: the state is untouched
        a.qout = static_cast<char*>(h->pq) + (size_t)zm_pq_elems(h->nx, h->ny, h->nz) * h->es;
        float tq = 1e30f, tl = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaError_t e = launch_zm(h, a);
          if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
          if (e != cudaSuccess) {
            destroy();
            return cuda_fail(e, "autotune");
          }
          float mq = 0.f, ml = 0.f;
          cudaEventElapsedTime(&mq, ev[0], ev[1]);
          cudaEventElapsedTime(&ml, ev[1], ev[2]);
          tq = std::min(tq, mq);
          tl = std::min(tl, ml);
        }
        if (tl < best_l) {
          best_l = tl;
          best_zc = zc;
          best_spt = spt;
        }
        if (tq < best_q) {
          best_q = tq;
          best_zq = zc;
          best_sq = sq;
        }
      }
    }
  }
  destroy();
  h->zc = best_zc;
  h->zc_q = best_zq;
  h->spt = best_spt;
  h->spt_q = best_sq;
  if (pinned) return LCBP_OK;
  g_tune[key] = {best_zc, best_spt + 10 * best_sq, best_zq};
  if (path) {
    if (FILE* fp = std::fopen(path, "a")) {
      std::fprintf(fp, "%s %d %d %d\n", key.c_str(), best_zc, best_spt + 10 * best_sq, best_zq);
      std::fclose(fp);
    }
  }
  return LCBP_OK;
}

int check_device_error(lcbp_lattice* h) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "error flag");
  if (flag) {
    cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    return fail(LCBP_ETIMEOUT, "a bounded device-side wait timed out; the step's results are not valid");
  }
  return LCBP_OK;
}

StepArgs step_args(lcbp_lattice* h) {
  StepArgs a{};
  a.reps = h->d_rep;
  a.tiles = h->d_tiles;
  a.ntiles = h->ntiles;
  a.ts = h->ts;
  a.flow_on = h->p.flow_on;
  a.coupling = h->p.coupling;
  a.walls = h->p.walls_z;
  a.div = h->p.l2_set && h->p.L2 != h->p.K;
  a.q = h->q;
  a.qs = h->qs;
  a.h = h->h;
  a.sigma = h->sig;
  a.tau = h->tau;
  a.b = h->b;
  a.bext = h->has_bext ? h->bext : nullptr;
  a.f = h->f[h->cur];
  a.fnew = h->f[h->cur ^ 1];
  a.rhou = h->rhou[h->cur];
  a.rhou_new = h->rhou[h->cur ^ 1];
  a.qout = nullptr;
  a.max_grid = 0;
  a.events = nullptr;
  return a;
}

cudaError_t eager_step(lcbp_lattice* h) {
  cudaError_t e;
  if (use_fast(h)) {
    const ModelBuf mb = host_model(h);
    e = launch_zm(h, zm_args(h, mb.bytes));
  } else {
    const StepArgs a = step_args(h);
    e = h->dtype == LCBP_F64 ? launch_step<double>(a, h->stream) : launch_step<float>(a, h->stream);
  }
  if (h->p.flow_on) h->cur ^= 1;
  return e;
}

void drop_graph(lcbp_lattice* h) {
  if (h->graph_ok) cudaGraphExecDestroy(h->graph);
  h->graph_ok = false;
}

// capture two steps starting from cur == 0 (the ping-pong buffers return to
// their roles after two steps)
int build_graph(lcbp_lattice* h) {
  if (h->stream == nullptr) return LCBP_OK;  // legacy stream: no capture, eager launches
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  const int saved = h->cur;
  h->cur = 0;
  cudaError_t e1 = eager_step(h);
  cudaError_t e2 = eager_step(h);
  h->cur = saved;
  e = cudaStreamEndCapture(h->stream, &g);
  if (e1 != cudaSuccess) e = e1;
  if (e2 != cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "graph capture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  h->graph_ok = true;
  return LCBP_OK;
}

int sync_flat(lcbp_lattice* h);

int diag(lcbp_lattice* h, double threshold, int with_f) {
  const int rs = sync_flat(h);
  if (rs) return rs;
  DiagGeom g{h->nx, h->ny, h->nz, h->n, 0, h->p.A0, h->p.gamma, h->p.K, h->p.q0, h->p.walls_z, {}, 0.0};
  for (int c = 0; c < 5; ++c) g.qw[c] = h->p.q_wall[c];
  g.c_div = h->p.l2_set ? 0.5 * (h->p.K - h->p.L2) : 0.0;
  cudaError_t e = h->dtype == LCBP_F64
                      ? launch_diag_one<double>(g, h->q, h->f[h->cur], with_f, threshold, h->d_partials, h->d_out,
                                                h->stream)
                      : launch_diag_one<float>(g, h->q, h->f[h->cur], with_f, threshold, h->d_partials, h->d_out,
                                               h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_out, h->d_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics");
  int rc = check_device_error(h);
  if (rc) return rc;
  if (h->h_out[6] != 0.0) return fail(LCBP_ENONFINITE, "%.0f sites hold NaN or Inf", h->h_out[6]);
  return LCBP_OK;
}

// number of non-finite values among n state-type values at v (device), synchronously
int count_nonfinite(lcbp_lattice* h, const void* v, long long n, unsigned long long* count) {
  auto* out = reinterpret_cast<unsigned long long*>(h->d_out);
  cudaError_t e = h->dtype == LCBP_F64 ? launch_count_nonfinite<double>(v, n, h->d_partials, out, h->stream)
                                       : launch_count_nonfinite<float>(v, n, h->d_partials, out, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_out, h->d_out, 8, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "finiteness check");
  *count = *reinterpret_cast<const unsigned long long*>(h->h_out);
  return LCBP_OK;
}

#define CHECK_H(h)                                                     \
  do {                                                                 \
    if (!(h)) return fail(LCBP_EINVAL, "null lattice handle");         \
    cudaSetDevice((h)->device);                                        \
  } while (0)

int refresh_moments(lcbp_lattice* h) {
  cudaError_t e = h->dtype == LCBP_F64
                      ? launch_moments<double>(h->d_rep, h->d_tiles, h->ntiles, h->ts, h->f[h->cur], h->rhou[h->cur],
                                               h->stream)
                      : launch_moments<float>(h->d_rep, h->d_tiles, h->ntiles, h->ts, h->f[h->cur], h->rhou[h->cur],
                                              h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "moments");
}

// The fast path keeps Q and rho u[cur] in padded mirrors with periodic
// ghosts (so its kernels stage them with no patching); every other kernel and
// every copy to or from the caller uses the flat arrays.  flat_ok / mirror_ok
// tell which copy is current (at least one is): fast steps make the mirrors
// current (sync_mirror before them), anything else reads or writes the flat
// arrays (sync_flat before, and a write makes the mirrors stale).
int sync_flat(lcbp_lattice* h) {
  if (h->flat_ok) return LCBP_OK;
  const int nxm = zm_mirror_nx(h->nx), X = kZmMirX;
  cudaError_t e =
      h->dtype == LCBP_F64
          ? launch_unpack<double>(h->qm, h->q, 5, 1, h->nx, h->ny, h->nz, X, 2, nxm, h->ny + 4, h->stream)
          : launch_unpack<float>(h->qm, h->q, 5, 1, h->nx, h->ny, h->nz, X, 2, nxm, h->ny + 4, h->stream);
  if (e == cudaSuccess)
    e = h->dtype == LCBP_F64
            ? launch_unpack<double>(h->um[h->cur], h->rhou[h->cur], 4, 1, h->nx, h->ny, h->nz, X, 1, nxm, h->ny + 2,
                                    h->stream)
            : launch_unpack<float>(h->um[h->cur], h->rhou[h->cur], 4, 1, h->nx, h->ny, h->nz, X, 1, nxm, h->ny + 2,
                                   h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "state from the padded mirrors");
  h->flat_ok = true;
  return LCBP_OK;
}

int sync_mirror(lcbp_lattice* h) {
  if (h->mirror_ok) return LCBP_OK;
  const int nxm = zm_mirror_nx(h->nx), X = kZmMirX;
  cudaError_t e = h->dtype == LCBP_F64
                      ? launch_pack<double>(h->q, h->qm, 5, 1, h->nx, h->ny, h->nz, X, 2, nxm, h->ny + 4, h->stream)
                      : launch_pack<float>(h->q, h->qm, 5, 1, h->nx, h->ny, h->nz, X, 2, nxm, h->ny + 4, h->stream);
  if (e == cudaSuccess)
    e = h->dtype == LCBP_F64
            ? launch_pack<double>(h->rhou[h->cur], h->um[h->cur], 4, 1, h->nx, h->ny, h->nz, X, 1, nxm, h->ny + 2,
                                  h->stream)
            : launch_pack<float>(h->rhou[h->cur], h->um[h->cur], 4, 1, h->nx, h->ny, h->nz, X, 1, nxm, h->ny + 2,
                                 h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "padded mirrors of the state");
  h->mirror_ok = true;
  return LCBP_OK;
}

struct CkptHeader {
  char magic[8];
  int32_t version, nx, ny, nz, dtype, flow_on, coupling, pad;
  double A0, gamma, K, q0, tau_f, xi, Gamma;
  int64_t step;
};
// version 3 appends the walls after the version-2 header
struct CkptWalls {
  int32_t walls_z, l2_set;
  double q_wall[5];
  double L2;
};

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

const char* lcbp_strerror(int code) {
  switch (code) {
    case LCBP_OK: return "LCBP_OK";
    case LCBP_EINVAL: return "LCBP_EINVAL: invalid argument";
    case LCBP_ENOMEM: return "LCBP_ENOMEM: out of memory";
    case LCBP_ECUDA: return "LCBP_ECUDA: CUDA error";
    case LCBP_ENONFINITE: return "LCBP_ENONFINITE: non-finite state";
    case LCBP_ETIMEOUT: return "LCBP_ETIMEOUT: device wait timed out";
    case LCBP_ESTATE: return "LCBP_ESTATE: call out of order";
    case LCBP_EIO: return "LCBP_EIO: checkpoint I/O failed";
    default: return "unknown lcbp status";
  }
}

const char* lcbp_last_error(void) { return g_last_error.c_str(); }

int lcbp_version(void) { return LCBP_VERSION; }

size_t lcbp_workspace_bytes(int nx, int ny, int nz, int dtype) {
  if (check_dims(nx, ny, nz) != LCBP_OK || !valid_dtype(dtype)) return 0;
  return layout(nx, ny, nz, dtype).total;
}

int lcbp_create(int nx, int ny, int nz, int dtype, lcbp_lattice** out) {
  if (!out) return fail(LCBP_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_dims(nx, ny, nz);
  if (rc) return rc;
  if (!valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad state dtype %d", dtype);
  lcbp_lattice* h = new_handle(nx, ny, nz, dtype);
  const Layout L = layout(nx, ny, nz, dtype);
  cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaStreamCreate");
  }
  h->own_stream = true;
  e = cudaMalloc(&h->ws, L.total);
  if (e != cudaSuccess) {
    cudaStreamDestroy(h->stream);
    delete h;
    cudaGetLastError();
    return fail(LCBP_ENOMEM, "cudaMalloc of %zu bytes failed", L.total);
  }
  h->own_ws = true;
  h->ws_bytes = L.total;
  rc = finish_create(h);
  if (rc) {
    lcbp_destroy(h);
    return rc;
  }
  *out = h;
  return LCBP_OK;
}

int lcbp_create_on_buffers(int nx, int ny, int nz, int dtype, void* workspace, size_t workspace_bytes, void* stream,
                           lcbp_lattice** out) {
  if (!out) return fail(LCBP_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_dims(nx, ny, nz);
  if (rc) return rc;
  if (!valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad state dtype %d", dtype);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return fail(LCBP_EINVAL, "workspace must be a 256-byte aligned device pointer");
  const Layout L = layout(nx, ny, nz, dtype);
  if (workspace_bytes < L.total)
    return fail(LCBP_ENOMEM, "workspace of %zu bytes, need %zu", workspace_bytes, L.total);
  lcbp_lattice* h = new_handle(nx, ny, nz, dtype);
  h->stream = static_cast<cudaStream_t>(stream);
  h->own_stream = false;
  h->ws = static_cast<char*>(workspace);
  h->ws_bytes = workspace_bytes;
  h->own_ws = false;
  rc = finish_create(h);
  if (rc) {
    lcbp_destroy(h);
    return rc;
  }
  *out = h;
  return LCBP_OK;
}

int lcbp_destroy(lcbp_lattice* h) {
  if (!h) return LCBP_OK;
  cudaSetDevice(h->device);
  if (h->stream || h->own_stream) cudaStreamSynchronize(h->stream);
  drop_graph(h);
  if (h->h_out) cudaFreeHost(h->h_out);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return LCBP_OK;
}

int lcbp_get_info(const lcbp_lattice* h, int dims[3], int* dtype, long long* step) {
  if (!h) return fail(LCBP_EINVAL, "null lattice handle");
  if (dims) {
    dims[0] = h->nx;
    dims[1] = h->ny;
    dims[2] = h->nz;
  }
  if (dtype) *dtype = h->dtype;
  if (step) *step = h->step;
  return LCBP_OK;
}

int lcbp_set_ldg(lcbp_lattice* h, double A0, double gamma, double K, double q0) {
  CHECK_H(h);
  HostParams p = h->p;
  p.A0 = A0;
  p.gamma = gamma;
  p.K = K;
  p.q0 = q0;
  int rc = check_params(p);
  if (rc) return rc;
  h->p = p;
  return upload_replica(h);
}

// gamma and K from the reduced chirality and temperature (Sec. 2.1)
static int ldg_from_kappa_tau(double A0, double q0, double kappa, double tau, double* gamma, double* K) {
  if (!(tau > -9.0) || q0 == 0.0 || !(kappa >= 0.0) || !std::isfinite(A0) || !std::isfinite(q0) ||
      !std::isfinite(kappa) || !std::isfinite(tau))
    return fail(LCBP_EINVAL, "need finite values, tau > -9, q0 != 0, kappa >= 0");
  *gamma = 27.0 / (9.0 + tau);
  *K = kappa * kappa * A0 * *gamma / (108.0 * q0 * q0);
  return LCBP_OK;
}

int lcbp_set_ldg_kappa_tau(lcbp_lattice* h, double A0, double q0, double kappa, double tau) {
  CHECK_H(h);
  double gamma = 0, K = 0;
  const int rc = ldg_from_kappa_tau(A0, q0, kappa, tau, &gamma, &K);
  return rc ? rc : lcbp_set_ldg(h, A0, gamma, K, q0);
}

int lcbp_params_kappa_tau(double A0, double q0, double kappa, double tau, double tau_f, double xi, double Gamma,
                          lcbp_params* out) {
  if (!out) return fail(LCBP_EINVAL, "out is NULL");
  double gamma = 0, K = 0;
  const int rc = ldg_from_kappa_tau(A0, q0, kappa, tau, &gamma, &K);
  if (rc) return rc;
  *out = lcbp_params{A0, gamma, K, q0, tau_f, xi, Gamma};
  return LCBP_OK;
}

size_t lcbp_snapshot_bytes(lcbp_lattice* h) { return h ? (size_t)(24 * h->n) * h->es : 0; }

int lcbp_snapshot(lcbp_lattice* h, void* dst) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!dst) return fail(LCBP_EINVAL, "dst is NULL");
  if (!h->f_ready) return fail(LCBP_ESTATE, "f was never initialised");
  const size_t nf = (size_t)(15 * h->n) * h->es, nr = (size_t)(4 * h->n) * h->es, nq = (size_t)(5 * h->n) * h->es;
  char* d = static_cast<char*>(dst);
  cudaError_t e = cudaMemcpyAsync(d, h->f[h->cur], nf, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + nf, h->rhou[h->cur], nr, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + nf + nr, h->q, nq, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "snapshot");
}

int lcbp_restore(lcbp_lattice* h, const void* src) {
  CHECK_H(h);
  if (!src) return fail(LCBP_EINVAL, "src is NULL");
  const size_t nf = (size_t)(15 * h->n) * h->es, nr = (size_t)(4 * h->n) * h->es, nq = (size_t)(5 * h->n) * h->es;
  const char* d = static_cast<const char*>(src);
  cudaError_t e = cudaMemcpyAsync(h->f[h->cur], d, nf, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->rhou[h->cur], d + nf, nr, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->q, d + nf + nr, nq, cudaMemcpyDefault, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "restore");
  h->f_ready = true;
  h->flat_ok = true;
  h->mirror_ok = false;
  return LCBP_OK;
}

int lcbp_set_flow(lcbp_lattice* h, double tau_f, double rho0, double xi, double Gamma, int flow_on, int coupling) {
  CHECK_H(h);
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail(LCBP_EINVAL, "need a finite rho0 > 0");
  HostParams p = h->p;
  p.rho0 = rho0;
  p.tau_f = tau_f;
  p.xi = xi;
  p.Gamma = Gamma;
  p.flow_on = flow_on ? 1 : 0;
  p.coupling = coupling;
  int rc = check_params(p);
  if (rc) return rc;
  if (p.flow_on != h->p.flow_on || p.coupling != h->p.coupling) drop_graph(h);
  h->p = p;
  return upload_replica(h);
}

int lcbp_set_l2(lcbp_lattice* h, int use_l2, double L2) {
  CHECK_H(h);
  if (use_l2 && !std::isfinite(L2)) return fail(LCBP_EINVAL, "L2 must be finite");
  if (use_l2 && h->p.walls_z) return fail(LCBP_EINVAL, "L2 with walls is not supported");
  HostParams p = h->p;
  p.l2_set = use_l2 ? 1 : 0;
  p.L2 = use_l2 ? L2 : 0.0;
  drop_graph(h);  // the fast path may no longer apply
  h->p = p;
  return upload_replica(h);
}

int lcbp_set_walls(lcbp_lattice* h, int walls_z, const double* q_wall5) {
  CHECK_H(h);
  if (walls_z && h->p.l2_set) return fail(LCBP_EINVAL, "walls with L2 are not supported");
  HostParams p = h->p;
  p.walls_z = walls_z ? 1 : 0;
  for (int c = 0; c < 5; ++c) {
    p.q_wall[c] = q_wall5 ? q_wall5[c] : 0.0;
    if (!std::isfinite(p.q_wall[c])) return fail(LCBP_EINVAL, "non-finite q_wall");
  }
  // the fast kernels take q_wall as a launch argument: recapture the step
  drop_graph(h);
  if (p.walls_z != h->p.walls_z) {
    h->zc = 0;  // tuned separately with walls
    h->spt = 0;
    h->spt_q = 0;
  }
  h->p = p;
  return upload_replica(h);
}

int lcbp_init_q(lcbp_lattice* h, int kind, double amplitude, double noise, uint64_t seed, const int* region) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  h->mirror_ok = false;  // the flat state is written below
  if (kind < LCBP_BPII || kind > LCBP_SLAB_BPII_IN_CHOL_Z) return fail(LCBP_EINVAL, "unknown initial kind %d", kind);
  if (!(noise >= 0.0) || !std::isfinite(amplitude)) return fail(LCBP_EINVAL, "need noise >= 0, finite amplitude");
  if (kind >= LCBP_SLAB_BPII_IN_CHOL && !region) return fail(LCBP_EINVAL, "slab kinds need region[0] = z0");
  InitQArgs a{kind, amplitude, noise, seed, region ? region[0] : 0};
  cudaError_t e = cudaMemcpyAsync(h->d_seed, &seed, sizeof(seed), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = h->dtype == LCBP_F64 ? launch_init_q<double>(h->d_rep, h->d_tiles, h->ntiles, h->ts, h->d_q0, h->d_shelix,
                                                     h->d_seed, a, h->q, h->stream)
                             : launch_init_q<float>(h->d_rep, h->d_tiles, h->ntiles, h->ts, h->d_q0, h->d_shelix,
                                                    h->d_seed, a, h->q, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "init_q");
}

int lcbp_set_q(lcbp_lattice* h, const void* q5, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  h->mirror_ok = false;  // the flat state is written below
  if (!q5 || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  // into the Q* scratch first: a field holding NaN or Inf is refused and Q stays as it was
  int rc = transfer(h->qs, h->dtype, const_cast<void*>(q5), dtype, 5 * h->n, true, h->staging, h->staging_elems,
                    h->stream);
  if (rc) return rc;
  unsigned long long bad = 0;
  rc = count_nonfinite(h, h->qs, 5 * h->n, &bad);
  if (rc) return rc;
  if (bad) return fail(LCBP_ENONFINITE, "%llu values of the uploaded Q are NaN or Inf; Q is unchanged", bad);
  cudaError_t e = cudaMemcpyAsync(h->q, h->qs, (size_t)(5 * h->n) * h->es, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "set_q");
}

int lcbp_init_f_equilibrium(lcbp_lattice* h, double rho0, const void* u3, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  h->mirror_ok = false;  // the flat state is written below
  if (rho0 == 0.0) rho0 = h->p.rho0;  // the lattice's reference density
  if (!(rho0 > 0.0) || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "need rho0 > 0 (or 0) and a valid dtype");
  int rc;
  if (u3) {
    // the body-force scratch holds the uploaded velocity
    rc = transfer(h->b, h->dtype, const_cast<void*>(u3), dtype, 3 * h->n, true, h->staging, h->staging_elems,
                  h->stream);
    if (rc) return rc;
  }
  StepArgs a = step_args(h);
  cudaError_t e = h->dtype == LCBP_F64 ? launch_field<double>(a, h->stream) : launch_field<float>(a, h->stream);
  if (e == cudaSuccess)
    e = h->dtype == LCBP_F64 ? launch_init_feq<double>(h->d_rep, h->d_tiles, h->ntiles, h->ts, rho0,
                                                       u3 ? h->b : nullptr, h->sig, h->f[h->cur], h->stream)
                             : launch_init_feq<float>(h->d_rep, h->d_tiles, h->ntiles, h->ts, rho0,
                                                      u3 ? h->b : nullptr, h->sig, h->f[h->cur], h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "init_f_equilibrium");
  rc = refresh_moments(h);
  if (rc) return rc;
  h->f_ready = true;
  return LCBP_OK;
}

int lcbp_set_f(lcbp_lattice* h, const void* f15, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  h->mirror_ok = false;  // the flat state is written below
  if (!f15 || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  // into the scratch block (16 N elements) first: non-finite populations are refused, f stays as it was
  int rc = transfer(h->h, h->dtype, const_cast<void*>(f15), dtype, 15 * h->n, true, h->staging, h->staging_elems,
                    h->stream);
  if (rc) return rc;
  unsigned long long bad = 0;
  rc = count_nonfinite(h, h->h, 15 * h->n, &bad);
  if (rc) return rc;
  if (bad) return fail(LCBP_ENONFINITE, "%llu uploaded populations are NaN or Inf; f is unchanged", bad);
  // into f as deviations from the rest weights, in one pass from the scratch
  cudaError_t e = h->dtype == LCBP_F64 ? launch_shift<double>(h->h, h->f[h->cur], h->n, 15, 0, -1, h->stream)
                                       : launch_shift<float>(h->h, h->f[h->cur], h->n, 15, 0, -1, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_f");
  rc = refresh_moments(h);
  if (rc) return rc;
  h->f_ready = true;
  return LCBP_OK;
}

int lcbp_set_body_force(lcbp_lattice* h, const void* b3, int dtype) {
  CHECK_H(h);
  if (!b3) {
    if (h->has_bext) drop_graph(h);
    h->has_bext = false;
    return LCBP_OK;
  }
  if (!valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad dtype");
  int rc = transfer(h->bext, h->dtype, const_cast<void*>(b3), dtype, 3 * h->n, true, h->staging, h->staging_elems,
                    h->stream);
  if (rc) return rc;
  if (!h->has_bext) drop_graph(h);
  h->has_bext = true;
  return LCBP_OK;
}

int lcbp_step(lcbp_lattice* h, int nsteps) {
  CHECK_H(h);
  if (nsteps < 0) return fail(LCBP_EINVAL, "nsteps < 0");
  if (h->p.flow_on && !h->f_ready) return fail(LCBP_ESTATE, "initialise f before stepping with flow on");
  if (nsteps == 0) return LCBP_OK;
  const bool fast = use_fast(h);
  {
    const int rs = fast ? sync_mirror(h) : sync_flat(h);
    if (rs) return rs;
  }
  if (fast && h->zc == 0) {
    int rc = tune_zc(h);
    if (rc) return rc;
  }
  // the kernel set's copy of the state is the one that changes
  if (fast) h->flat_ok = false;
  else h->mirror_ok = false;
  cudaError_t e = cudaSuccess;
  int left = nsteps;
  if (h->cur == 1) {
    e = eager_step(h);
    --left;
  }
  if (left >= 2 && !h->graph_ok && e == cudaSuccess) {
    int rc = build_graph(h);
    if (rc) return rc;
  }
  while (left >= 2 && e == cudaSuccess) {
    if (h->graph_ok) {
      e = cudaGraphLaunch(h->graph, h->stream);
    } else {
      e = eager_step(h);
      if (e == cudaSuccess) e = eager_step(h);
    }
    left -= 2;
  }
  if (left == 1 && e == cudaSuccess) e = eager_step(h);
  if (e != cudaSuccess) return cuda_fail(e, "step launch");
  h->step += nsteps;
  return LCBP_OK;
}

int lcbp_profile_steps(lcbp_lattice* h, int nsteps, double* kernel_ms, int capacity, int* nkernels) {
  CHECK_H(h);
  if (nsteps < 1 || !kernel_ms || !nkernels) return fail(LCBP_EINVAL, "need nsteps >= 1 and output arrays");
  if (h->p.flow_on && !h->f_ready) return fail(LCBP_ESTATE, "initialise f before stepping with flow on");
  const bool fast = use_fast(h);
  {
    const int rs = fast ? sync_mirror(h) : sync_flat(h);
    if (rs) return rs;
  }
  if (fast && h->zc == 0) {
    int rc = tune_zc(h);
    if (rc) return rc;
  }
  if (fast) h->flat_ok = false;
  else h->mirror_ok = false;
  const int nk = fast ? 2 : kernels_per_step(h->p.flow_on, h->p.coupling);
  *nkernels = nk;
  if (capacity < nk) return fail(LCBP_EINVAL, "kernel_ms holds %d values, need %d", capacity, nk);
  std::vector<cudaEvent_t> ev((size_t)nsteps * (nk + 1));
  cudaError_t e = cudaSuccess;
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreate(&x);
  for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
    if (fast) {
      const ModelBuf mb = host_model(h);
      ZmArgs a = zm_args(h, mb.bytes);
      a.events = ev.data() + (size_t)s * (nk + 1);
      e = launch_zm(h, a);
    } else {
      StepArgs a = step_args(h);
      a.events = ev.data() + (size_t)s * (nk + 1);
      e = h->dtype == LCBP_F64 ? launch_step<double>(a, h->stream) : launch_step<float>(a, h->stream);
    }
    if (h->p.flow_on) h->cur ^= 1;
    h->step += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  for (int k = 0; k < nk; ++k) kernel_ms[k] = 0.0;
  for (int s = 0; s < nsteps && e == cudaSuccess; ++s)
    for (int k = 0; k < nk && e == cudaSuccess; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[(size_t)s * (nk + 1) + k], ev[(size_t)s * (nk + 1) + k + 1]);
      kernel_ms[k] += ms / nsteps;
    }
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return cuda_fail(e, "profile_steps");
  return check_device_error(h);
}

int lcbp_set_path(lcbp_lattice* h, int path) {
  CHECK_H(h);
  if (path < LCBP_PATH_AUTO || path > LCBP_PATH_FAST2) return fail(LCBP_EINVAL, "unknown path %d", path);
  if (path == LCBP_PATH_FAST2 && h->dtype == LCBP_F64)
    return fail(LCBP_EINVAL, "two sites per thread exist for FP32 lattices only");
  drop_graph(h);
  h->path_req = path;
  h->zc = 0;  // retune for the new choice
  h->spt = 0;
  h->spt_q = 0;
  return LCBP_OK;
}

int lcbp_get_tuning(lcbp_lattice* h, int* planes_per_cta, int* spt_lb, int* spt_q, int* planes_per_cta_q) {
  CHECK_H(h);
  const bool f = use_fast(h) && h->zc > 0;
  if (planes_per_cta) *planes_per_cta = f ? h->zc : 0;
  if (planes_per_cta_q) *planes_per_cta_q = f ? (h->zc_q > 0 ? h->zc_q : h->zc) : 0;
  if (spt_lb) *spt_lb = f ? h->spt : 0;
  if (spt_q) *spt_q = f ? (h->spt_q > 0 ? h->spt_q : h->spt) : 0;
  return LCBP_OK;
}

int lcbp_get_path(lcbp_lattice* h, int* fast, int* planes_per_cta, int* sites_per_thread) {
  CHECK_H(h);
  const bool f = use_fast(h);
  if (fast) *fast = f ? 1 : 0;
  if (planes_per_cta) *planes_per_cta = f ? h->zc : 0;
  if (sites_per_thread) *sites_per_thread = f && h->zc > 0 ? h->spt : 0;
  return LCBP_OK;
}

int lcbp_synchronize(lcbp_lattice* h) {
  CHECK_H(h);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  return check_device_error(h);
}

int lcbp_check_wait_timeout(double limit_ms, int* timed_out) {
  if (!timed_out || !(limit_ms > 0.0 && limit_ms <= 1000.0))
    return fail(LCBP_EINVAL, "need 0 < limit_ms <= 1000 and an output");
  int* d_flag = nullptr;
  cudaError_t e = cudaMalloc(&d_flag, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemset(d_flag, 0xff, sizeof(int));
  if (e == cudaSuccess) e = launch_wait_probe((uint64_t)(limit_ms * 1e6), d_flag, nullptr);
  int flag = -1;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_flag);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (flag != 0 && flag != 1) return fail(LCBP_ECUDA, "wait self-test: the probe did not report");
  *timed_out = flag;
  return LCBP_OK;
}

int lcbp_read_q(lcbp_lattice* h, void* dst, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  return transfer(h->q, h->dtype, dst, dtype, 5 * h->n, false, h->staging, h->staging_elems, h->stream);
}

int lcbp_read_u(lcbp_lattice* h, void* dst, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  return transfer(static_cast<char*>(h->rhou[h->cur]) + h->n * h->es, h->dtype, dst, dtype, 3 * h->n, false,
                  h->staging, h->staging_elems, h->stream);
}

int lcbp_read_rho(lcbp_lattice* h, void* dst, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  // rho = 1 + drho, assembled in the (free between steps) predictor scratch
  cudaError_t e = h->dtype == LCBP_F64 ? launch_shift<double>(h->rhou[h->cur], h->qs, h->n, 1, 1, 1, h->stream)
                                       : launch_shift<float>(h->rhou[h->cur], h->qs, h->n, 1, 1, 1, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "read_rho");
  return transfer(h->qs, h->dtype, dst, dtype, h->n, false, h->staging, h->staging_elems, h->stream);
}

int lcbp_read_f(lcbp_lattice* h, void* dst, int dtype) {
  CHECK_H(h);
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  // f = w + df, assembled in the other ping-pong buffer (free between steps)
  void* tmp = h->f[h->cur ^ 1];
  cudaError_t e = h->dtype == LCBP_F64 ? launch_shift<double>(h->f[h->cur], tmp, h->n, 15, 0, 1, h->stream)
                                       : launch_shift<float>(h->f[h->cur], tmp, h->n, 15, 0, 1, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "read_f");
  return transfer(tmp, h->dtype, dst, dtype, 15 * h->n, false, h->staging, h->staging_elems, h->stream);
}

int lcbp_free_energy(lcbp_lattice* h, double* F) {
  CHECK_H(h);
  if (!F) return fail(LCBP_EINVAL, "F is NULL");
  int rc = diag(h, 0.0, 0);
  if (rc) return rc;
  *F = h->h_out[0];
  return LCBP_OK;
}

int lcbp_totals(lcbp_lattice* h, double* mass, double momentum[3]) {
  CHECK_H(h);
  int rc = diag(h, 0.0, 1);
  if (rc) return rc;
  if (mass) *mass = h->h_out[1];
  if (momentum) {
    momentum[0] = h->h_out[2];
    momentum[1] = h->h_out[3];
    momentum[2] = h->h_out[4];
  }
  return LCBP_OK;
}

int lcbp_defect_fraction(lcbp_lattice* h, double threshold, double* fraction) {
  CHECK_H(h);
  if (!fraction) return fail(LCBP_EINVAL, "fraction is NULL");
  int rc = diag(h, threshold, 0);
  if (rc) return rc;
  *fraction = h->h_out[5] / (double)h->n;
  return LCBP_OK;
}

int lcbp_texture(lcbp_lattice* h, const lcbp_optics* o, float* img) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!o || !img) return fail(LCBP_EINVAL, "o and img must not be NULL");
  if (o->nlambda < 1 || o->nlambda > 4) return fail(LCBP_EINVAL, "nlambda must be 1..4, got %d", o->nlambda);
  for (int l = 0; l < o->nlambda; ++l)
    if (!(o->lambda[l] > 0)) return fail(LCBP_EINVAL, "wavelength %d must be > 0", l);
  // the H scratch (5 N elements) is free between steps and holds the image
  // and the per-split column products
  float* d_img = static_cast<float*>(h->h);
  const long long scratch = 5LL * h->n * dtype_size(h->dtype) / (long long)sizeof(float);
  cudaError_t e = h->dtype == LCBP_F64
                      ? launch_texture<double>(h->q, h->nx, h->ny, h->nz, *o, d_img, scratch, h->stream)
                      : launch_texture<float>(h->q, h->nx, h->ny, h->nz, *o, d_img, scratch, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(img, d_img, sizeof(float) * (size_t)h->nx * h->ny, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "texture");
  return LCBP_OK;
}

// Checkpoints hold the raw state (deviation populations, moments, Q) in the
// state type, so that a resumed run is bitwise identical to an uninterrupted one.
int lcbp_save(lcbp_lattice* h, const char* path) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!path) return fail(LCBP_EINVAL, "path is NULL");
  CkptHeader hd{};
  std::memcpy(hd.magic, "LCBPCKP2", 8);
  hd.version = 3;
  CkptWalls wl{};
  wl.walls_z = h->p.walls_z;
  for (int c = 0; c < 5; ++c) wl.q_wall[c] = h->p.q_wall[c];
  wl.l2_set = h->p.l2_set;
  wl.L2 = h->p.L2;
  hd.nx = h->nx;
  hd.ny = h->ny;
  hd.nz = h->nz;
  hd.dtype = h->dtype;
  hd.flow_on = h->p.flow_on;
  hd.coupling = h->p.coupling;
  hd.A0 = h->p.A0;
  hd.gamma = h->p.gamma;
  hd.K = h->p.K;
  hd.q0 = h->p.q0;
  hd.tau_f = h->p.tau_f;
  hd.xi = h->p.xi;
  hd.Gamma = h->p.Gamma;
  hd.step = h->step;
  const size_t nf = (size_t)15 * h->n * h->es, nr = (size_t)4 * h->n * h->es, nq = (size_t)5 * h->n * h->es;
  std::vector<char> buf(nf + nr + nq);
  cudaError_t e = cudaMemcpyAsync(buf.data(), h->f[h->cur], nf, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf.data() + nf, h->rhou[h->cur], nr, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf.data() + nf + nr, h->q, nq, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "save");
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(LCBP_EIO, "cannot open %s for writing", path);
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(&wl, sizeof(wl), 1, fp) == 1 &&
                  std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
  const bool closed = std::fclose(fp) == 0;
  return ok && closed ? LCBP_OK : fail(LCBP_EIO, "short write to %s", path);
}

int lcbp_load(lcbp_lattice* h, const char* path) {
  CHECK_H(h);
  if (!path) return fail(LCBP_EINVAL, "path is NULL");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(LCBP_EIO, "cannot open %s", path);
  CkptHeader hd{};
  if (std::fread(&hd, sizeof(hd), 1, fp) != 1 || std::memcmp(hd.magic, "LCBPCKP2", 8) != 0 ||
      (hd.version != 2 && hd.version != 3)) {
    std::fclose(fp);
    return fail(LCBP_EIO, "%s is not an lcbp checkpoint", path);
  }
  CkptWalls wl{};  // version 2 files have no walls
  if (hd.version == 3 && std::fread(&wl, sizeof(wl), 1, fp) != 1) {
    std::fclose(fp);
    return fail(LCBP_EIO, "truncated checkpoint %s", path);
  }
  if (hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz || hd.dtype != h->dtype) {
    std::fclose(fp);
    return fail(LCBP_EINVAL, "checkpoint dims/dtype do not match the lattice");
  }
  const size_t nf = (size_t)15 * h->n * h->es, nr = (size_t)4 * h->n * h->es, nq = (size_t)5 * h->n * h->es;
  std::vector<char> buf(nf + nr + nq);
  const bool ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
  std::fclose(fp);
  if (!ok) return fail(LCBP_EIO, "truncated checkpoint %s", path);
  HostParams p = h->p;
  p.A0 = hd.A0;
  p.gamma = hd.gamma;
  p.K = hd.K;
  p.q0 = hd.q0;
  p.tau_f = hd.tau_f;
  p.xi = hd.xi;
  p.Gamma = hd.Gamma;
  p.flow_on = hd.flow_on;
  p.coupling = hd.coupling;
  p.walls_z = wl.walls_z;
  for (int c = 0; c < 5; ++c) p.q_wall[c] = wl.q_wall[c];
  p.l2_set = wl.l2_set;
  p.L2 = wl.L2;
  int rc = check_params(p);
  if (rc) return rc;
  if (p.flow_on != h->p.flow_on || p.coupling != h->p.coupling || p.walls_z != h->p.walls_z ||
      p.l2_set != h->p.l2_set || p.L2 != h->p.L2)
    drop_graph(h);
  h->p = p;
  rc = upload_replica(h);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(h->f[h->cur], buf.data(), nf, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->rhou[h->cur], buf.data() + nf, nr, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->q, buf.data() + nf + nr, nq, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "load");
  h->f_ready = true;
  h->flat_ok = true;
  h->mirror_ok = false;
  h->step = hd.step;
  return LCBP_OK;
}

int lcbp_read_rate(lcbp_lattice* h, void* dst, int dtype) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  if (h->p.flow_on && !h->f_ready) return fail(LCBP_ESTATE, "initialise f first (u comes from f)");
  StepArgs a = step_args(h);
  cudaError_t e = h->dtype == LCBP_F64 ? launch_rate<double>(a, h->stream) : launch_rate<float>(a, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "read_rate");
  return transfer(h->qs, h->dtype, dst, dtype, 5 * h->n, false, h->staging, h->staging_elems, h->stream);
}

int lcbp_reequilibrate_f(lcbp_lattice* h) {
  CHECK_H(h);
  {
    const int rs = sync_flat(h);
    if (rs) return rs;
  }
  h->mirror_ok = false;  // the flat state is written below
  if (!h->f_ready) return fail(LCBP_ESTATE, "f was never initialised");
  StepArgs a = step_args(h);
  cudaError_t e = h->dtype == LCBP_F64 ? launch_field<double>(a, h->stream) : launch_field<float>(a, h->stream);
  if (e == cudaSuccess)
    e = h->dtype == LCBP_F64 ? launch_feq_from_moments<double>(h->d_rep, h->d_tiles, h->ntiles, h->ts,
                                                                h->rhou[h->cur], h->sig, h->f[h->cur], h->stream)
                             : launch_feq_from_moments<float>(h->d_rep, h->d_tiles, h->ntiles, h->ts,
                                                               h->rhou[h->cur], h->sig, h->f[h->cur], h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reequilibrate_f");
  return refresh_moments(h);
}

}  // extern "C"

namespace lcbp {
// Enqueue the Beris-Edwards rate of a lattice into its predictor scratch on
// the lattice's stream and record `done` after it; returns that scratch
// (5 * N floats, valid until the lattice's next step)
int lattice_rate(lcbp_lattice* h, const float** rate, cudaEvent_t done) {
  if (!h) return fail(LCBP_EINVAL, "null lattice handle");
  if (h->dtype != LCBP_F32) return fail(LCBP_EINVAL, "the surrogate works on FP32 lattice state");
  cudaSetDevice(h->device);
  const int rs = sync_flat(h);
  if (rs) return rs;
  StepArgs a = step_args(h);
  cudaError_t e = launch_rate<float>(a, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(done, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rate");
  *rate = static_cast<const float*>(h->qs);
  return LCBP_OK;
}

int lattice_fields(lcbp_lattice* h, float** q, const float** u, int dims[3], cudaStream_t* stream) {
  if (!h) return fail(LCBP_EINVAL, "null lattice handle");
  if (h->dtype != LCBP_F32) return fail(LCBP_EINVAL, "the surrogate works on FP32 lattice state");
  if (h->p.walls_z) return fail(LCBP_EINVAL, "the surrogate's convolutions are periodic: no walls");
  cudaSetDevice(h->device);
  const int rs = sync_flat(h);
  if (rs) return rs;
  h->mirror_ok = false;  // the surrogate updates Q in place
  *q = static_cast<float*>(h->q);
  *u = reinterpret_cast<const float*>(static_cast<const char*>(h->rhou[h->cur]) + h->n * sizeof(float));
  dims[0] = h->nx;
  dims[1] = h->ny;
  dims[2] = h->nz;
  *stream = h->stream;
  return LCBP_OK;
}

// a new lattice of the same dims, dtype, parameters and kernel-set choice
// (state unset): the surrogate judge's scratch lattice
int lattice_clone(lcbp_lattice* src, lcbp_lattice** out) {
  if (!src || !out) return fail(LCBP_EINVAL, "null lattice handle");
  cudaSetDevice(src->device);
  int rc = lcbp_create(src->nx, src->ny, src->nz, src->dtype, out);
  if (rc) return rc;
  lcbp_lattice* d = *out;
  d->p = src->p;
  d->path_req = src->path_req;
  rc = upload_replica(d);
  if (rc) {
    lcbp_destroy(d);
    *out = nullptr;
  }
  return rc;
}

// device Q (5 N state-type values, updated in place by steps) and the stream
int lattice_q(lcbp_lattice* h, const void** q, long long* n, int* dtype, cudaStream_t* stream) {
  if (!h) return fail(LCBP_EINVAL, "null lattice handle");
  cudaSetDevice(h->device);
  const int rs = sync_flat(h);
  if (rs) return rs;
  *q = h->q;
  *n = h->n;
  *dtype = h->dtype;
  *stream = h->stream;
  return LCBP_OK;
}
}  // namespace lcbp
