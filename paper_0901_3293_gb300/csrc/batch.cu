// Batched replicas: R lattices of uneven sizes and per-replica parameters
// stepped together.  Fields are concatenated structure-of-arrays blocks
// (replica r of a C-component field at field + C * base_r, laid out
// [c][z][y][x]); replicas of equal dims (a class) are stored back to back.
//
// Two step paths, both one launch per kernel over every replica and replayed
// from a captured CUDA graph:
// * fast (flow on, Jacobi coupling, every class with nx % 4 = 0, at most
//   kZmMaxClasses classes): the z-marching TMA kernels, each field of a class
//   read as one 5-D tensor (x, y, z, component, replica); the planes per CTA
//   are chosen by timing candidates on the batch (scratch outputs only);
// * generic: one tile work-list spans every replica and the one-site-per-
//   thread kernels run as persistent CTAs; the tile shape is chosen by timing
//   candidate shapes on the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lcbp.h"
#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

using namespace lcbp;

struct lcbp_batch {
  int R;
  int dtype;
  size_t es;
  int device;
  std::vector<int> nx, ny, nz;
  std::vector<long long> n, base;
  long long ntot;
  std::vector<HostParams> p;
  int flow_on, coupling;
  cudaStream_t stream;
  char* ws;
  void *f[2], *rhou[2], *q, *qs, *h, *sig, *tau, *b, *staging;
  void* pq;  // the fast kernels' padded scratch, class by class (overlays h, sig, tau, b)
  // the fast kernels' state: padded mirrors of Q and rho u (two buffers),
  // class by class, and a Q mirror the tuner writes; the flat fields and the
  // mirrors are kept in step lazily (flat_ok / mirror_ok)
  void *qm, *qm_tune, *um[2];
  bool flat_ok, mirror_ok;
  long long staging_elems;
  void* d_rep;
  Tile* d_tiles;
  long long tile_cap;
  int ntiles;
  std::vector<int> tile_begin;  // per replica, + end
  TileShape ts;
  bool tuned;
  int max_grid;
  double *d_q0, *d_shelix, *d_partials, *d_out, *h_out;
  uint64_t* d_seed;
  int cur;
  bool f_ready;
  cudaGraphExec_t graph;
  bool graph_ok;
  long long step;
  // fast path
  std::vector<int> order;  // replica indices class by class, in storage order
  ZmBatch zb;              // classes (zc and CTA ranges filled when tuned) for k_lbq_batch
  ZmBatch zbq;             // the same classes with k_qside_batch's planes per CTA
  ZmBatchMaps maps[2];     // tensor maps with rho u buffer 0 / 1
  bool fast_ok;            // every class fits the fast kernels
  bool fast_pick;          // AUTO: the fast kernels timed faster than the generic ones
  int path_req;            // LCBP_PATH_AUTO, LCBP_PATH_GENERIC or LCBP_PATH_FAST1
  int zc;                  // planes per CTA (0 = not tuned)
  int* d_order;
  int* d_err;
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr long long kStaging = 1ll << 22;

const TileShape kCandidates[] = {{32, 4, 1}, {32, 2, 2}, {16, 8, 1}, {16, 4, 2}, {32, 8, 1}, {8, 8, 2}, {32, 1, 4}};

int check_b(lcbp_batch* b) {
  if (!b) return fail(LCBP_EINVAL, "null batch handle");
  cudaSetDevice(b->device);
  return LCBP_OK;
}

int check_r(lcbp_batch* b, int r) {
  if (r < 0 || r >= b->R) return fail(LCBP_EINVAL, "replica %d out of range [0, %d)", r, b->R);
  return LCBP_OK;
}

void drop_graph(lcbp_batch* b) {
  if (b->graph_ok) cudaGraphExecDestroy(b->graph);
  b->graph_ok = false;
}

bool fast_eligible(const lcbp_batch* b) {
  return b->fast_ok && b->path_req != LCBP_PATH_GENERIC && b->flow_on && b->coupling == LCBP_JACOBI;
}

bool use_fast(const lcbp_batch* b) {
  return fast_eligible(b) && (b->path_req == LCBP_PATH_FAST1 || b->fast_pick);
}

// Tensor maps of every class, the replica outermost (replicas of a class back
// to back): the Q mirrors as their [xx xy xz yy] vectors and their yz arrays
// (replica stride 5 cq), the rho u mirrors (stride 4 cu) and the padded
// scratch (stride 16 (nx+4)(ny+2)nz)
bool build_maps(lcbp_batch* b) {
  for (int k = 0; k < b->zb.nclass; ++k) {
    const ZmClass& c = b->zb.c[k];
    // boxes of the class's tiles (tx x ty sites): Q tx + 8 wide from x0 - 4, ty + 4 rows; rho u and the
    // scratch tx + 2 wide from x0 - 1, ty + 2 rows
    const int tx = c.G.tx, ty = c.G.ty;
    const cuuint64_t es = b->es;
    const cuuint64_t nx = c.G.nx, ny = c.G.ny, nz = c.G.nz;
    const cuuint64_t nxm = zm_mirror_nx(c.G.nx), nyq = ny + 4, nyu = ny + 2, cq = nxm * nyq * nz, cu = nxm * nyu * nz;
    // a plane-interleaved mirror array [replica][nz][nym][w] with replica stride rs elements
    auto mirror = [&](CUtensorMap* tm, void* arr, long long off, cuuint64_t w, cuuint64_t nym, cuuint64_t rs,
                      int inner, int rows) {
      const cuuint64_t dims[4] = {w, nym, nz, (cuuint64_t)c.count};
      const cuuint64_t strides[3] = {w * es, w * nym * es, rs * es};
      const cuuint32_t box[4] = {(cuuint32_t)inner, (cuuint32_t)rows, 1, 1};
      return encode_tiled(tm, static_cast<char*>(arr) + (size_t)off * es, 4, dims, strides, box, b->dtype);
    };
    const cuuint64_t nxp = nx + kZmPadX, nyp = ny + 2, cp = nxp * nyp * nz;
    // the scratch [replica][z][group][Y][X][4] as (4 X, Y, group, z, replica)
    const cuuint64_t pdims[5] = {4 * nxp, nyp, (cuuint64_t)kZmPQG, nz, (cuuint64_t)c.count};
    const cuuint64_t pstr[4] = {4 * nxp * es, 4 * nxp * nyp * es, (cuuint64_t)kZmPQ * nxp * nyp * es,
                                (cuuint64_t)kZmPQ * cp * es};
    const cuuint32_t pbox[5] = {(cuuint32_t)(4 * (tx + 2)), (cuuint32_t)(ty + 2), (cuuint32_t)kZmPQG, 1, 1};
    bool ok = mirror(&b->maps[0].q[k], b->qm, c.qm0, 4 * nxm, nyq, 5 * cq, 4 * (tx + 8), ty + 4) &&
              mirror(&b->maps[0].q1[k], b->qm, c.qm0 + 4 * (long long)cq, nxm, nyq, 5 * cq, tx + 8, ty + 4) &&
              mirror(&b->maps[0].u[k], b->um[0], c.um0, 4 * nxm, nyu, 4 * cu, 4 * (tx + 2), ty + 2) &&
              mirror(&b->maps[1].u[k], b->um[1], c.um0, 4 * nxm, nyu, 4 * cu, 4 * (tx + 2), ty + 2) &&
              encode_tiled(&b->maps[0].pq[k], static_cast<char*>(b->pq) + (size_t)c.pq0 * b->es, 5, pdims, pstr,
                           pbox, b->dtype);
    // k_lbq's L2 prefetches: the Q mirrors in tile-sized boxes, and the flat
    // populations of the class's replicas (blocks of NV * round64(n) elements)
    // in boxes of the tile's rows (all populations) or of one halo row (one or
    // two populations)
    ok = ok && mirror(&b->maps[0].qpf[k], b->qm, c.qm0, 4 * nxm, nyq, 5 * cq, 4 * tx, ty) &&
         mirror(&b->maps[0].q1pf[k], b->qm, c.qm0 + 4 * (long long)cq, nxm, nyq, 5 * cq, tx, ty);
    const cuuint64_t rstride = (cuuint64_t)NV * ((c.G.n + 63) / 64 * 64);
    const cuuint64_t fdims[5] = {nx, ny, nz, (cuuint64_t)NV, (cuuint64_t)c.count};
    const cuuint64_t fstr[4] = {nx * es, nx * ny * es, nx * ny * nz * es, rstride * es};
    const cuuint32_t fbox[5] = {(cuuint32_t)(tx + 8), (cuuint32_t)ty, 1, (cuuint32_t)NV, 1};
    const cuuint32_t fbox1[5] = {(cuuint32_t)(tx + 8), 1, 1, 1, 1}, fbox2[5] = {(cuuint32_t)(tx + 8), 1, 1, 2, 1};
    for (int j = 0; j < 2 && ok; ++j) {
      char* fb = static_cast<char*>(b->f[j]) + (size_t)NV * b->base[b->order[c.rep0]] * es;  // first replica
      ok = encode_tiled(&b->maps[j].f[k], fb, 5, fdims, fstr, fbox, b->dtype) &&
           encode_tiled(&b->maps[j].f1[k], fb, 5, fdims, fstr, fbox1, b->dtype) &&
           encode_tiled(&b->maps[j].f2[k], fb, 5, fdims, fstr, fbox2, b->dtype);
    }
    if (!ok) return false;
    b->maps[1].qpf[k] = b->maps[0].qpf[k];
    b->maps[1].q1pf[k] = b->maps[0].q1pf[k];
    b->maps[0].u3[k] = b->maps[0].u[k];
    b->maps[1].u3[k] = b->maps[1].u[k];
    b->maps[1].q[k] = b->maps[0].q[k];
    b->maps[1].q1[k] = b->maps[0].q1[k];
    b->maps[1].pq[k] = b->maps[0].pq[k];
  }
  return true;
}

// geometry and CTA ranges of the classes of zb for zc[k] planes per CTA in class k
void fill_zc(ZmBatch& zb, const int* zc) {
  int cta = 0;
  for (int k = 0; k < zb.nclass; ++k) {
    ZmClass& c = zb.c[k];
    c.G.zc = std::min(zc[k], c.G.nz);
    c.G.tiles_x = (c.G.nx + c.G.tx - 1) / c.G.tx;
    c.G.tiles_y = (c.G.ny + c.G.ty - 1) / c.G.ty;
    c.G.tiles_z = (c.G.nz + c.G.zc - 1) / c.G.zc;
    c.ctas_per_rep = c.G.tiles_x * c.G.tiles_y * c.G.tiles_z;
    c.G.nxp = c.G.nx + kZmPadX;
    c.G.nyp = c.G.ny + 2;
    c.G.cp = (long long)c.G.nxp * c.G.nyp * c.G.nz;
    c.G.nxm = zm_mirror_nx(c.G.nx);
    c.G.nyq = c.G.ny + 4;
    c.G.nyu = c.G.ny + 2;
    c.G.cq = (long long)c.G.nxm * c.G.nyq * c.G.nz;
    c.G.cu = (long long)c.G.nxm * c.G.nyu * c.G.nz;
    c.cta0 = cta;
    cta += c.ctas_per_rep * c.count;
  }
  zb.total_ctas = cta;
}

// planes per CTA of each class for k_lbq_batch (zc) and k_qside_batch (zc_q)
void set_zc(lcbp_batch* b, const int* zc, const int* zc_q) {
  fill_zc(b->zb, zc);
  b->zbq = b->zb;
  fill_zc(b->zbq, zc_q);
  b->zc = zc[0];
}

ZmBatchArgs zm_args(lcbp_batch* b) {
  ZmBatchArgs a{};
  a.B = b->zb;
  a.Bq = b->zbq;
  a.maps = &b->maps[b->cur];
  a.reps = b->d_rep;
  a.order = b->d_order;
  a.q = b->qm;
  a.qout = nullptr;
  a.pq = b->pq;
  a.f = b->f[b->cur];
  a.fnew = b->f[b->cur ^ 1];
  a.rhou = b->um[b->cur];
  a.rhou_new = b->um[b->cur ^ 1];
  a.err = b->d_err;
  return a;
}

// Q and rho u (the current buffer) of every replica of the fast-path classes,
// between the flat fields and the padded mirrors: unpack (mirrors -> flat) or
// pack (flat -> mirrors, periodic images included)
cudaError_t mirror_copy(lcbp_batch* b, bool to_flat) {
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < b->zb.nclass && e == cudaSuccess; ++k) {
    const ZmClass& c = b->zb.c[k];
    const int nx = c.G.nx, ny = c.G.ny, nz = c.G.nz, nxm = zm_mirror_nx(nx), X = kZmMirX;
    const long long cq = (long long)nxm * (ny + 4) * nz, cu = (long long)nxm * (ny + 2) * nz;
    for (int j = 0; j < c.count && e == cudaSuccess; ++j) {
      const int r = b->order[c.rep0 + j];
      char* qm = static_cast<char*>(b->qm) + (size_t)(c.qm0 + j * 5 * cq) * b->es;
      char* um = static_cast<char*>(b->um[b->cur]) + (size_t)(c.um0 + j * 4 * cu) * b->es;
      void* q = static_cast<char*>(b->q) + (size_t)5 * b->base[r] * b->es;
      void* ru = static_cast<char*>(b->rhou[b->cur]) + (size_t)4 * b->base[r] * b->es;
      const bool d = b->dtype == LCBP_F64;
      if (to_flat) {
        e = d ? launch_unpack<double>(qm, q, 5, 1, nx, ny, nz, X, 2, nxm, ny + 4, b->stream)
              : launch_unpack<float>(qm, q, 5, 1, nx, ny, nz, X, 2, nxm, ny + 4, b->stream);
        if (e == cudaSuccess)
          e = d ? launch_unpack<double>(um, ru, 4, 1, nx, ny, nz, X, 1, nxm, ny + 2, b->stream)
                : launch_unpack<float>(um, ru, 4, 1, nx, ny, nz, X, 1, nxm, ny + 2, b->stream);
      } else {
        e = d ? launch_pack<double>(q, qm, 5, 1, nx, ny, nz, X, 2, nxm, ny + 4, b->stream)
              : launch_pack<float>(q, qm, 5, 1, nx, ny, nz, X, 2, nxm, ny + 4, b->stream);
        if (e == cudaSuccess)
          e = d ? launch_pack<double>(ru, um, 4, 1, nx, ny, nz, X, 1, nxm, ny + 2, b->stream)
                : launch_pack<float>(ru, um, 4, 1, nx, ny, nz, X, 1, nxm, ny + 2, b->stream);
      }
    }
  }
  return e;
}

// the flat fields current (readers, writers and the generic kernels)
int sync_flat(lcbp_batch* b) {
  if (b->flat_ok) return LCBP_OK;
  const cudaError_t e = mirror_copy(b, true);
  if (e != cudaSuccess) return cuda_fail(e, "mirror unpack");
  b->flat_ok = true;
  return LCBP_OK;
}

// the mirrors current (the fast kernels)
int sync_mirror(lcbp_batch* b) {
  if (b->mirror_ok || !b->fast_ok) return LCBP_OK;
  const cudaError_t e = mirror_copy(b, false);
  if (e != cudaSuccess) return cuda_fail(e, "mirror pack");
  b->mirror_ok = true;
  return LCBP_OK;
}

cudaError_t launch_zm(lcbp_batch* b, const ZmBatchArgs& a) {
  return b->dtype == LCBP_F64 ? launch_step_zm_batch<double>(a, b->stream)
                              : launch_step_zm_batch<float>(a, b->stream);
}

int check_error_flag(lcbp_batch* b) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "error flag");
  if (flag) {
    cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
    return fail(LCBP_ETIMEOUT, "a bounded device-side wait timed out; the step's results are not valid");
  }
  return LCBP_OK;
}

int build_tiles(lcbp_batch* b, TileShape ts) {
  std::vector<Tile> tiles;
  b->tile_begin.assign(b->R + 1, 0);
  for (int r = 0; r < b->R; ++r) {
    b->tile_begin[r] = (int)tiles.size();
    // every replica uses the same shape: the kernels map threads by it
    append_tiles(tiles, r, b->nx[r], b->ny[r], b->nz[r], ts);
  }
  b->tile_begin[b->R] = (int)tiles.size();
  if ((long long)tiles.size() > b->tile_cap) return fail(LCBP_ENOMEM, "tile list overflow");
  b->ntiles = (int)tiles.size();
  b->ts = ts;
  cudaError_t e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "tile upload");
}

int upload_table(lcbp_batch* b) {
  drop_graph(b);
  const size_t rb = replica_bytes(b->dtype);
  std::vector<char> buf(rb * b->R);
  std::vector<double> aux(2 * b->R);
  for (int r = 0; r < b->R; ++r) {
    if (b->dtype == LCBP_F64)
      fill_replica<double>(buf.data() + rb * r, b->nx[r], b->ny[r], b->nz[r], b->base[r], b->p[r]);
    else
      fill_replica<float>(buf.data() + rb * r, b->nx[r], b->ny[r], b->nz[r], b->base[r], b->p[r]);
    aux[r] = b->p[r].q0;
    aux[b->R + r] = s_eq(b->p[r].gamma);
  }
  cudaError_t e = cudaMemcpyAsync(b->d_rep, buf.data(), buf.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_q0, aux.data(), b->R * 8, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_shelix, aux.data() + b->R, b->R * 8, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "replica table upload");
}

StepArgs args(lcbp_batch* b) {
  StepArgs a{};
  a.reps = b->d_rep;
  a.tiles = b->d_tiles;
  a.ntiles = b->ntiles;
  a.ts = b->ts;
  a.flow_on = b->flow_on;
  a.coupling = b->coupling;
  a.q = b->q;
  a.qs = b->qs;
  a.h = b->h;
  a.sigma = b->sig;
  a.tau = b->tau;
  a.b = b->b;
  a.bext = nullptr;
  a.f = b->f[b->cur];
  a.fnew = b->f[b->cur ^ 1];
  a.rhou = b->rhou[b->cur];
  a.rhou_new = b->rhou[b->cur ^ 1];
  a.qout = nullptr;
  a.max_grid = b->max_grid;
  a.events = nullptr;
  return a;
}

cudaError_t launch(lcbp_batch* b, const StepArgs& a) {
  return b->dtype == LCBP_F64 ? launch_step<double>(a, b->stream) : launch_step<float>(a, b->stream);
}

cudaError_t eager(lcbp_batch* b) {
  const cudaError_t e = use_fast(b) ? launch_zm(b, zm_args(b)) : launch(b, args(b));
  if (b->flow_on) b->cur ^= 1;
  return e;
}

// persistent grid: as many CTAs as can be resident at once
int resident_ctas(lcbp_batch* b) {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = b->ts.tx * b->ts.ty * b->ts.tz;
  // 128-register kernels: at most 65536 / (threads * 128) CTAs per SM
  const int per_sm = std::max(1, 65536 / (threads * 128));
  return std::max(1, sms * per_sm);
}

// planes per CTA of the fast path, per class and per kernel: one value for
// every class first, then each class's own value with the others held (one
// pass); every candidate is one step of the whole batch (best of 3) with an
// event between the kernels, and each kernel keeps its own best values (the
// kernels run one after the other, so their times add)
int tune_fast(lcbp_batch* b, float* best_ms) {
  cudaEvent_t ev[3];
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(LCBP_ECUDA, "events");
  const int nc = b->zb.nclass;
  const int cand[] = {4, 6, 8, 10, 12, 16, 24, 32, 48, 64};
  cudaError_t err = cudaSuccess;
  // time of k_qside_batch with zc_q and of k_lbq_batch with zc (best of 3 each)
  auto time_zc = [&](const int* zc, const int* zc_q, float* tq, float* tl) {
    set_zc(b, zc, zc_q);
    ZmBatchArgs a = zm_args(b);
    a.qout = b->qm_tune;  // a mirror the state does not use: the state is left untouched
    a.events = ev;
    *tq = *tl = 1e30f;
    for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
      err = launch_zm(b, a);
      if (err == cudaSuccess) err = cudaEventSynchronize(ev[2]);
      float m0 = 0, m1 = 0;
      if (err == cudaSuccess) {
        cudaEventElapsedTime(&m0, ev[0], ev[1]);
        cudaEventElapsedTime(&m1, ev[1], ev[2]);
      }
      *tq = std::min(*tq, m0);
      *tl = std::min(*tl, m1);
    }
  };
  int zl[kZmMaxClasses], zq[kZmMaxClasses], best_l[kZmMaxClasses], best_q[kZmMaxClasses];
  float bl = 1e30f, bq = 1e30f;
  int max_nz = 1;
  for (int k = 0; k < nc; ++k) max_nz = std::max(max_nz, b->zb.c[k].G.nz);
  for (int v : cand) {
    if (v > max_nz && v != 4) break;
    for (int k = 0; k < nc; ++k) zl[k] = zq[k] = v;
    float tq, tl;
    time_zc(zl, zq, &tq, &tl);
    if (tl < bl) {
      bl = tl;
      std::copy(zl, zl + nc, best_l);
    }
    if (tq < bq) {
      bq = tq;
      std::copy(zq, zq + nc, best_q);
    }
  }
  for (int k = 0; k < nc && nc > 1 && err == cudaSuccess; ++k) {
    std::copy(best_l, best_l + nc, zl);
    std::copy(best_q, best_q + nc, zq);
    const int hold_l = best_l[k], hold_q = best_q[k];
    for (int v : cand) {
      if (v > b->zb.c[k].G.nz && v != 4) break;
      if (v == hold_l && v == hold_q) continue;
      zl[k] = zq[k] = v;
      float tq, tl;
      time_zc(zl, zq, &tq, &tl);
      if (tl < bl) {
        bl = tl;
        best_l[k] = v;
      }
      if (tq < bq) {
        bq = tq;
        best_q[k] = v;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return cuda_fail(err, "batch planes-per-CTA tuning");
  set_zc(b, best_l, best_q);
  *best_ms = bl + bq;
  return check_error_flag(b);
}

// tile shape of the generic path: timed candidates, one step each (best of 3)
int tune_generic(lcbp_batch* b, float* best_ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(LCBP_ECUDA, "events");
  float best = 1e30f;
  TileShape best_ts = kCandidates[0];
  for (const TileShape& c : kCandidates) {
    int rc = build_tiles(b, c);
    if (rc) return rc;
    b->max_grid = resident_ctas(b);
    StepArgs a = args(b);
    a.qout = b->h;  // scratch: the state is left untouched
    float t = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, b->stream);
      cudaError_t e = launch(b, a);
      cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return cuda_fail(e, "tile tuning");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t = std::min(t, ms);
    }
    if (t < best) {
      best = t;
      best_ts = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc = build_tiles(b, best_ts);
  if (rc) return rc;
  b->max_grid = resident_ctas(b);
  *best_ms = best;
  return LCBP_OK;
}

// Tune the path the batch will run; with LCBP_PATH_AUTO and both paths open,
// tune both and keep the faster.
int tune(lcbp_batch* b) {
  float t_fast = 1e30f, t_gen = 1e30f;
  int rc = sync_flat(b);  // the generic tuner reads the flat fields, the fast one the mirrors
  if (!rc && fast_eligible(b)) rc = sync_mirror(b);
  if (fast_eligible(b)) rc = tune_fast(b, &t_fast);
  if (!rc && (!fast_eligible(b) || b->path_req == LCBP_PATH_AUTO)) rc = tune_generic(b, &t_gen);
  if (rc) return rc;
  b->fast_pick = t_fast < t_gen;
  b->tuned = true;
  return LCBP_OK;
}

int build_graph(lcbp_batch* b) {
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "capture");
  const int saved = b->cur;
  b->cur = 0;
  cudaError_t e1 = eager(b);
  cudaError_t e2 = eager(b);
  b->cur = saved;
  e = cudaStreamEndCapture(b->stream, &g);
  if (e1 != cudaSuccess) e = e1;
  if (e2 != cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "capture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "instantiate");
  b->graph_ok = true;
  return LCBP_OK;
}

void* field(lcbp_batch* b, void* arr, int comps, int r) {
  return static_cast<char*>(arr) + (size_t)comps * b->base[r] * b->es;
}

int moments_all(lcbp_batch* b) {
  cudaError_t e = b->dtype == LCBP_F64 ? launch_moments<double>(b->d_rep, b->d_tiles, b->ntiles, b->ts,
                                                                b->f[b->cur], b->rhou[b->cur], b->stream)
                                       : launch_moments<float>(b->d_rep, b->d_tiles, b->ntiles, b->ts, b->f[b->cur],
                                                               b->rhou[b->cur], b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "moments");
}

int diag(lcbp_batch* b, int r, double threshold, int with_f) {
  const int rs = sync_flat(b);
  if (rs) return rs;
  DiagGeom g{b->nx[r], b->ny[r], b->nz[r], b->n[r], b->base[r], b->p[r].A0, b->p[r].gamma, b->p[r].K, b->p[r].q0};
  cudaError_t e = b->dtype == LCBP_F64 ? launch_diag_one<double>(g, b->q, b->f[b->cur], with_f, threshold,
                                                                 b->d_partials, b->d_out, b->stream)
                                       : launch_diag_one<float>(g, b->q, b->f[b->cur], with_f, threshold,
                                                                b->d_partials, b->d_out, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_out, b->d_out, 64, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics");
  int rc = check_error_flag(b);
  if (rc) return rc;
  if (b->h_out[6] != 0.0) return fail(LCBP_ENONFINITE, "replica %d: %.0f sites hold NaN or Inf", r, b->h_out[6]);
  return LCBP_OK;
}

}  // namespace

extern "C" {

int lcbp_batch_create(int R, const int* dims, const lcbp_params* params, int dtype, lcbp_batch** out) {
  if (!out) return fail(LCBP_EINVAL, "out is NULL");
  *out = nullptr;
  if (R < 1 || !dims || !params) return fail(LCBP_EINVAL, "need R >= 1, dims and params");
  if (!valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad dtype");
  auto* b = new lcbp_batch();
  b->R = R;
  b->dtype = dtype;
  b->es = dtype_size(dtype);
  cudaGetDevice(&b->device);
  long long tot = 0, cap = 0;
  for (int r = 0; r < R; ++r) {
    const int x = dims[3 * r], y = dims[3 * r + 1], z = dims[3 * r + 2];
    if (x < 1 || y < 1 || z < 1) {
      delete b;
      return fail(LCBP_EINVAL, "replica %d has a size < 1", r);
    }
    b->nx.push_back(x);
    b->ny.push_back(y);
    b->nz.push_back(z);
    const long long n = (long long)x * y * z;
    b->n.push_back(n);
    long long mx = 0;
    for (const TileShape& c : kCandidates) mx = std::max(mx, tile_count(x, y, z, c));
    cap += mx;
    HostParams hp{};
    hp.A0 = params[r].A0;
    hp.gamma = params[r].gamma;
    hp.K = params[r].K;
    hp.q0 = params[r].q0;
    hp.tau_f = params[r].tau_f;
    hp.xi = params[r].xi;
    hp.Gamma = params[r].Gamma;
    hp.flow_on = 1;
    hp.coupling = LCBP_JACOBI;
    int rc = check_params(hp);
    if (rc) {
      delete b;
      return rc;
    }
    b->p.push_back(hp);
  }
  // classes of equal dims, in order of first appearance; storage class by class
  b->zb = ZmBatch{};
  b->fast_ok = true;
  std::vector<int> cls(R, -1);
  std::vector<std::vector<int>> members;
  for (int r = 0; r < R; ++r) {
    for (int k = 0; k < (int)members.size() && cls[r] < 0; ++k) {
      const int q = members[k][0];
      if (b->nx[q] == b->nx[r] && b->ny[q] == b->ny[r] && b->nz[q] == b->nz[r]) cls[r] = k;
    }
    if (cls[r] < 0) {
      cls[r] = (int)members.size();
      members.emplace_back();
    }
    members[cls[r]].push_back(r);
  }
  b->base.assign(R, 0);
  for (int k = 0; k < (int)members.size(); ++k) {
    const int q = members[k][0];
    if (k < kZmMaxClasses) {
      ZmClass& c = b->zb.c[k];
      c.G.nx = b->nx[q];
      c.G.ny = b->ny[q];
      c.G.nz = b->nz[q];
      c.G.n = b->n[q];
      // tile shape of the fast kernels: 32 x TY, or narrow 16 x 2 TY
      const int ty = dtype == LCBP_F64 ? zm_tile_rows<double>() : zm_tile_rows<float>();
      c.G.tx = zm_batch_tile_x(c.G.nx, dtype != LCBP_F64);
      c.G.ty = c.G.tx == kZmNarrowX ? 2 * ty : ty;
      c.rep0 = (int)b->order.size();
      c.count = (int)members[k].size();
    }
    if (!zm_shape_ok(b->nx[q], b->ny[q], b->nz[q])) b->fast_ok = false;
    for (int r : members[k]) {
      b->order.push_back(r);
      b->base[r] = tot;
      tot += (b->n[r] + 63) / 64 * 64;  // 256-byte aligned replica blocks in FP32
    }
  }
  if ((int)members.size() > kZmMaxClasses) b->fast_ok = false;
  b->zb.nclass = std::min((int)members.size(), kZmMaxClasses);
  // the fast kernels' padded scratch, class by class (64-element aligned blocks)
  long long pq_tot = 0;
  for (int k = 0; k < b->zb.nclass; ++k) {
    ZmClass& c = b->zb.c[k];
    c.pq0 = pq_tot;
    pq_tot += ((long long)c.count * zm_pq_elems(c.G.nx, c.G.ny, c.G.nz) + 63) / 64 * 64;
  }
  // the fast path's mirrors of Q and rho u, class by class (64-element aligned blocks)
  long long qm_tot = 0, um_tot = 0;
  for (int k = 0; k < b->zb.nclass && b->fast_ok; ++k) {
    ZmClass& c = b->zb.c[k];
    const long long nxm = zm_mirror_nx(c.G.nx), cq = nxm * (c.G.ny + 4) * c.G.nz, cu = nxm * (c.G.ny + 2) * c.G.nz;
    c.qm0 = qm_tot;
    qm_tot += ((long long)c.count * 5 * cq + 63) / 64 * 64;
    c.um0 = um_tot;
    um_tot += ((long long)c.count * 4 * cu + 63) / 64 * 64;
  }
  b->flat_ok = true;
  b->mirror_ok = false;
  b->path_req = LCBP_PATH_AUTO;
  b->fast_pick = true;
  b->zc = 0;
  if (tot > (1ll << 31)) {
    delete b;
    return fail(LCBP_EINVAL, "more than 2^31 sites");
  }
  b->ntot = tot;
  b->tile_cap = cap;
  b->flow_on = 1;
  b->coupling = LCBP_JACOBI;
  // f0 f1 rhou0 rhou1 q qs, then h sig tau b back to back in one block that
  // the fast kernels' padded scratch overlays (the two kernel sets never run
  // within one step, and no scratch outlives a step)
  const long long comps[6] = {15, 15, 4, 4, 5, 5};
  size_t off[10], o = 0;
  for (int i = 0; i < 6; ++i) {
    off[i] = o;
    o = a256(o + (size_t)comps[i] * tot * b->es);
  }
  off[6] = o;
  off[7] = o + (size_t)5 * tot * b->es;
  off[8] = o + (size_t)10 * tot * b->es;
  off[9] = o + (size_t)13 * tot * b->es;
  o = a256(o + (size_t)std::max(16 * tot, pq_tot) * b->es);
  const size_t off_stage = o;
  b->staging_elems = std::min(kStaging, 15 * tot);
  o = a256(o + (size_t)b->staging_elems * 8);
  const size_t off_rep = o;
  o = a256(o + replica_bytes(dtype) * R);
  const size_t off_tiles = o;
  o = a256(o + (size_t)cap * sizeof(Tile));
  const size_t off_aux = o;
  o = a256(o + (size_t)R * 3 * 8);
  const size_t off_part = o;
  o = a256(o + (kDiagPartials + 8) * 8);
  const size_t off_order = o;
  o = a256(o + (size_t)R * sizeof(int) + sizeof(int));
  size_t off_mir[4];
  for (int i = 0; i < 4; ++i) {  // Q mirrors, the tuner's Q mirrors, rho u mirrors 0 and 1
    off_mir[i] = o;
    o = a256(o + (size_t)(i < 2 ? qm_tot : um_tot) * b->es);
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->ws, o);
  if (e != cudaSuccess) {
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    cudaGetLastError();
    return fail(LCBP_ENOMEM, "batch allocation of %zu bytes failed", o);
  }
  char* w = b->ws;
  b->f[0] = w + off[0];
  b->f[1] = w + off[1];
  b->rhou[0] = w + off[2];
  b->rhou[1] = w + off[3];
  b->q = w + off[4];
  b->qs = w + off[5];
  b->h = w + off[6];
  b->sig = w + off[7];
  b->tau = w + off[8];
  b->b = w + off[9];
  b->pq = w + off[6];
  b->staging = w + off_stage;
  b->d_rep = w + off_rep;
  b->d_tiles = reinterpret_cast<Tile*>(w + off_tiles);
  b->d_q0 = reinterpret_cast<double*>(w + off_aux);
  b->d_shelix = b->d_q0 + R;
  b->d_seed = reinterpret_cast<uint64_t*>(b->d_q0 + 2 * R);
  b->d_partials = reinterpret_cast<double*>(w + off_part);
  b->d_out = b->d_partials + kDiagPartials;
  b->d_order = reinterpret_cast<int*>(w + off_order);
  b->qm = w + off_mir[0];
  b->qm_tune = w + off_mir[1];
  b->um[0] = w + off_mir[2];
  b->um[1] = w + off_mir[3];
  b->d_err = b->d_order + R;
  e = cudaMemsetAsync(b->ws, 0, off_stage, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_order, b->order.data(), (size_t)R * sizeof(int), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, 64);
  int rc = e == cudaSuccess ? LCBP_OK : cuda_fail(e, "batch set-up");
  if (!rc) rc = upload_table(b);
  if (!rc) rc = build_tiles(b, kCandidates[0]);
  if (!rc) b->max_grid = resident_ctas(b);
  if (!rc && b->fast_ok) {
    static std::once_flag prep32, prep64;
    if (dtype == LCBP_F64) std::call_once(prep64, [] { zm_batch_prepare<double>(); });
    else std::call_once(prep32, [] { zm_batch_prepare<float>(); });
    b->fast_ok = build_maps(b);  // no tensor maps: the generic kernels serve the batch
  }
  if (rc) {
    lcbp_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LCBP_OK;
}

int lcbp_batch_destroy(lcbp_batch* b) {
  if (!b) return LCBP_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->ws) cudaFree(b->ws);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LCBP_OK;
}

int lcbp_batch_set_flow(lcbp_batch* b, int flow_on, int coupling) {
  int rc = check_b(b);
  if (rc) return rc;
  if (coupling != LCBP_JACOBI && coupling != LCBP_GAUSS_SEIDEL) return fail(LCBP_EINVAL, "bad coupling");
  drop_graph(b);
  const bool was_open = fast_eligible(b);
  b->flow_on = flow_on ? 1 : 0;
  b->coupling = coupling;
  if (fast_eligible(b) != was_open) b->tuned = false;
  return LCBP_OK;
}

int lcbp_batch_set_path(lcbp_batch* b, int path) {
  int rc = check_b(b);
  if (rc) return rc;
  if (path != LCBP_PATH_AUTO && path != LCBP_PATH_GENERIC && path != LCBP_PATH_FAST1)
    return fail(LCBP_EINVAL, "a batch takes LCBP_PATH_AUTO, LCBP_PATH_GENERIC or LCBP_PATH_FAST1, got %d", path);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  b->path_req = path;
  b->tuned = false;
  return LCBP_OK;
}

int lcbp_batch_get_path(lcbp_batch* b, int* fast, int* planes_per_cta) {
  int rc = check_b(b);
  if (rc) return rc;
  const bool f = use_fast(b);
  if (fast) *fast = f ? 1 : 0;
  if (planes_per_cta) *planes_per_cta = f && b->tuned ? b->zc : 0;
  return LCBP_OK;
}

int lcbp_batch_init_q(lcbp_batch* b, int r, int kind, double amplitude, double noise, uint64_t seed,
                      const int* region) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  if (kind < LCBP_BPII || kind > LCBP_SLAB_BPII_IN_CHOL_Z) return fail(LCBP_EINVAL, "unknown initial kind %d", kind);
  if (!(noise >= 0.0)) return fail(LCBP_EINVAL, "noise < 0");
  if (kind >= LCBP_SLAB_BPII_IN_CHOL && !region) return fail(LCBP_EINVAL, "slab kinds need region");
  rc = sync_flat(b);  // the other replicas' flat Q stays current
  if (rc) return rc;
  b->mirror_ok = false;
  InitQArgs a{kind, amplitude, noise, seed, region ? region[0] : 0};
  cudaError_t e = cudaMemcpyAsync(b->d_seed + r, &seed, 8, cudaMemcpyHostToDevice, b->stream);
  const Tile* t0 = b->d_tiles + b->tile_begin[r];
  const int nt = b->tile_begin[r + 1] - b->tile_begin[r];
  if (e == cudaSuccess)
    e = b->dtype == LCBP_F64
            ? launch_init_q<double>(b->d_rep, t0, nt, b->ts, b->d_q0, b->d_shelix, b->d_seed, a, b->q, b->stream)
            : launch_init_q<float>(b->d_rep, t0, nt, b->ts, b->d_q0, b->d_shelix, b->d_seed, a, b->q, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "batch init_q");
}

int lcbp_batch_set_q(lcbp_batch* b, int r, const void* q5, int dtype) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  if (!q5 || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  rc = sync_flat(b);
  if (rc) return rc;
  b->mirror_ok = false;
  return transfer(field(b, b->q, 5, r), b->dtype, const_cast<void*>(q5), dtype, 5 * b->n[r], true, b->staging,
                  b->staging_elems, b->stream);
}

int lcbp_batch_init_f_equilibrium(lcbp_batch* b, double rho0) {
  int rc = check_b(b);
  if (rc) return rc;
  if (!(rho0 > 0)) return fail(LCBP_EINVAL, "rho0 <= 0");
  rc = sync_flat(b);
  if (rc) return rc;
  b->mirror_ok = false;
  StepArgs a = args(b);
  cudaError_t e = b->dtype == LCBP_F64 ? launch_field<double>(a, b->stream) : launch_field<float>(a, b->stream);
  if (e == cudaSuccess)
    e = b->dtype == LCBP_F64 ? launch_init_feq<double>(b->d_rep, b->d_tiles, b->ntiles, b->ts, rho0, nullptr,
                                                       b->sig, b->f[b->cur], b->stream)
                             : launch_init_feq<float>(b->d_rep, b->d_tiles, b->ntiles, b->ts, rho0, nullptr, b->sig,
                                                      b->f[b->cur], b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch init_f");
  rc = moments_all(b);
  if (rc) return rc;
  b->f_ready = true;
  return LCBP_OK;
}

int lcbp_batch_step(lcbp_batch* b, int nsteps) {
  int rc = check_b(b);
  if (rc) return rc;
  if (nsteps < 0) return fail(LCBP_EINVAL, "nsteps < 0");
  if (b->flow_on && !b->f_ready) return fail(LCBP_ESTATE, "initialise f before stepping with flow on");
  if (nsteps == 0) return LCBP_OK;
  if (!b->tuned) {
    rc = tune(b);
    if (rc) return rc;
    drop_graph(b);
  }
  const bool fast = use_fast(b);
  rc = fast ? sync_mirror(b) : sync_flat(b);
  if (rc) return rc;
  if (fast) b->flat_ok = false;
  else b->mirror_ok = false;
  cudaError_t e = cudaSuccess;
  int left = nsteps;
  if (b->cur == 1) {
    e = eager(b);
    --left;
  }
  if (left >= 2 && !b->graph_ok && e == cudaSuccess) {
    rc = build_graph(b);
    if (rc) return rc;
  }
  while (left >= 2 && e == cudaSuccess) {
    e = cudaGraphLaunch(b->graph, b->stream);
    left -= 2;
  }
  if (left == 1 && e == cudaSuccess) e = eager(b);
  if (e != cudaSuccess) return cuda_fail(e, "batch step");
  b->step += nsteps;
  return LCBP_OK;
}

int lcbp_batch_synchronize(lcbp_batch* b) {
  int rc = check_b(b);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  return check_error_flag(b);
}

int lcbp_batch_read_q(lcbp_batch* b, int r, void* dst, int dtype) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  rc = sync_flat(b);
  if (rc) return rc;
  return transfer(field(b, b->q, 5, r), b->dtype, dst, dtype, 5 * b->n[r], false, b->staging, b->staging_elems,
                  b->stream);
}

int lcbp_batch_read_u(lcbp_batch* b, int r, void* dst, int dtype) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  if (!dst || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffer or dtype");
  rc = sync_flat(b);
  if (rc) return rc;
  void* u = static_cast<char*>(field(b, b->rhou[b->cur], 4, r)) + b->n[r] * b->es;
  return transfer(u, b->dtype, dst, dtype, 3 * b->n[r], false, b->staging, b->staging_elems, b->stream);
}

int lcbp_batch_free_energy(lcbp_batch* b, int r, double* F) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  if (!F) return fail(LCBP_EINVAL, "F is NULL");
  rc = diag(b, r, 0.0, 0);
  if (rc) return rc;
  *F = b->h_out[0];
  return LCBP_OK;
}

int lcbp_batch_totals(lcbp_batch* b, int r, double* mass, double momentum[3]) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  rc = diag(b, r, 0.0, 1);
  if (rc) return rc;
  if (mass) *mass = b->h_out[1];
  if (momentum) {
    momentum[0] = b->h_out[2];
    momentum[1] = b->h_out[3];
    momentum[2] = b->h_out[4];
  }
  return LCBP_OK;
}

int lcbp_batch_defect_fraction(lcbp_batch* b, int r, double threshold, double* fraction) {
  int rc = check_b(b);
  if (!rc) rc = check_r(b, r);
  if (rc) return rc;
  if (!fraction) return fail(LCBP_EINVAL, "fraction is NULL");
  rc = diag(b, r, threshold, 0);
  if (rc) return rc;
  *fraction = b->h_out[5] / (double)b->n[r];
  return LCBP_OK;
}

int lcbp_batch_get_info(lcbp_batch* b, int* R, long long* total_sites, int tile[3], int* persistent_ctas,
                        long long* step) {
  int rc = check_b(b);
  if (rc) return rc;
  if (R) *R = b->R;
  if (total_sites) {
    long long s = 0;
    for (long long v : b->n) s += v;
    *total_sites = s;
  }
  if (tile) {
    tile[0] = b->ts.tx;
    tile[1] = b->ts.ty;
    tile[2] = b->ts.tz;
  }
  if (persistent_ctas) *persistent_ctas = b->max_grid;
  if (step) *step = b->step;
  return LCBP_OK;
}

}  // extern "C"
