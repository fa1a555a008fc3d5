// Judged surrogate run: the learned surrogate advances a lattice, and the
// plain solver judges it and takes over where it fails.
//
// The lattice advances in segments of M surrogate calls (k solver steps
// each, k of the surrogate).  A segment starts from a raw device snapshot of (f, rho u, Q).  After
// its calls f is re-equilibrated to the new Q, and the judge compares one more
// surrogate call with k plain steps from that same state: the relative gap
// of the free energy F_h (and, if asked, the largest |Delta Q|).  Within the
// tolerances the segment stands and the k plain steps count as time
// advanced; otherwise the snapshot is restored and the segment is redone with
// plain steps.  Free energy and defect fraction are logged at every multiple
// of a log interval, from the state the run actually keeps (a rolled-back
// segment's surrogate values are discarded and taken again from its plain
// redo).  Everything numerical runs in the library's kernels; this file only
// orders the calls.  The paper has no surrogate; the solver it judges by is
// the coupled step of Sec. 2.2.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/lcbp.h"
#include "kernels.h"
#include "runtime.h"

namespace lcbp {
int lattice_clone(lcbp_lattice* src, lcbp_lattice** out);
int lattice_q(lcbp_lattice* h, const void** q, long long* n, int* dtype, cudaStream_t* stream);
}  // namespace lcbp

using namespace lcbp;


struct lcbp_judge {
  long long k;  // solver steps one surrogate call stands for
  lcbp_lattice* lat;
  lcbp_surrogate* sur;
  lcbp_judge_config c;
  lcbp_lattice* scratch;  // the judge's copy of the state for its one surrogate call
  void* snap;             // segment start (device)
  void* snap2;            // state handed to the scratch lattice (device)
  void* red;              // reduction scratch for max |Delta Q| (device)
  double* h_red;          // pinned result
  lcbp_judge_stats st;
  // log entries of the current segment, kept only if the segment stands
  std::vector<long long> pt;
  std::vector<double> pF, pD;
};

namespace {

int jfail_cuda(cudaError_t e, const char* what) { return cuda_fail(e, what); }

// F_h and the defect fraction of the judged lattice
int measure(lcbp_judge* j, double thr, double* F, double* D) {
  int rc = lcbp_free_energy(j->lat, F);
  if (!rc) rc = lcbp_defect_fraction(j->lat, thr, D);
  return rc;
}

// Plain steps from t0 to t0 + n, logging at every multiple of log_every on the way
int plain(lcbp_judge* j, long long t0, long long n, int log_every, double thr, std::vector<long long>& lt,
          std::vector<double>& lF, std::vector<double>& lD) {
  long long t = t0;
  while (t < t0 + n) {
    long long chunk = t0 + n - t;
    if (log_every > 0) chunk = std::min(chunk, (t / log_every + 1) * (long long)log_every - t);
    int rc = lcbp_step(j->lat, (int)chunk);
    if (rc) return rc;
    t += chunk;
    j->st.plain_steps += chunk;
    if (log_every > 0 && t % log_every == 0) {
      double F = 0, D = 0;
      rc = measure(j, thr, &F, &D);
      if (rc) return rc;
      lt.push_back(t);
      lF.push_back(F);
      lD.push_back(D);
    }
  }
  return LCBP_OK;
}

}  // namespace

namespace {

// A library error inside a segment's surrogate part or its judgement fails
// the judgement when it reports a non-finite state; any other error ends the
// run with that status.
struct Soft {
  int hard = LCBP_OK;
  bool operator()(int rc) {
    if (rc == LCBP_OK) return true;
    if (rc != LCBP_ENONFINITE && hard == LCBP_OK) hard = rc;
    return false;
  }
};

// max |Q_scratch - Q_lattice| (both synchronised by the free-energy calls before)
int q_gap(lcbp_judge* j, double* gap) {
  const void *qa = nullptr, *qb = nullptr;
  long long n = 0, nb = 0;
  int da = 0, db = 0;
  cudaStream_t sa, sb;
  int rc = lattice_q(j->scratch, &qa, &n, &da, &sa);
  if (!rc) rc = lattice_q(j->lat, &qb, &nb, &db, &sb);
  if (rc) return rc;
  double* out = reinterpret_cast<double*>(static_cast<char*>(j->red) + state_check_scratch_bytes());
  cudaError_t e = da == LCBP_F64 ? launch_max_abs_diff<double>(qa, qb, 5 * n, j->red, out, sb)
                                 : launch_max_abs_diff<float>(qa, qb, 5 * n, j->red, out, sb);
  if (e == cudaSuccess) e = cudaMemcpyAsync(j->h_red, out, sizeof(double), cudaMemcpyDeviceToHost, sb);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sb);
  if (e != cudaSuccess) return jfail_cuda(e, "judge: max |dQ|");
  *gap = *j->h_red;
  return LCBP_OK;
}

// One segment of `calls` surrogate calls from time t.  *accepted tells
// whether it stood; the segment's log entries are in j->pt/pF/pD either way
// (a rolled-back segment's are those of its plain redo).
int segment(lcbp_judge* j, long long t, int calls, int log_every, double thr, bool* accepted) {
  j->pt.clear();
  j->pF.clear();
  j->pD.clear();
  int rc = lcbp_snapshot(j->lat, j->snap);
  if (rc) return rc;
  Soft soft;
  bool ok = true;
  int done = 0;
  while (ok && done < calls) {
    const long long tt = t + done * j->k;
    int n = calls - done;
    if (log_every > 0) n = (int)std::min<long long>(n, ((tt / log_every + 1) * log_every - tt) / j->k);
    ok = soft(lcbp_surrogate_step(j->sur, j->lat, j->c.kappa, j->c.tau, n));
    done += n;
    const long long te = t + done * j->k;
    if (ok && log_every > 0 && te % log_every == 0) {
      double F = 0, D = 0;
      ok = soft(measure(j, thr, &F, &D));
      j->pt.push_back(te);
      j->pF.push_back(F);
      j->pD.push_back(D);
    }
  }
  // the judgement: one surrogate call on a copy of the state against ten plain steps
  double Fs = 0, Fp = 0, gF = NAN, gQ = NAN;
  ok = ok && soft(lcbp_reequilibrate_f(j->lat));
  ok = ok && soft(lcbp_snapshot(j->lat, j->snap2)) && soft(lcbp_restore(j->scratch, j->snap2));
  ok = ok && soft(lcbp_surrogate_step(j->sur, j->scratch, j->c.kappa, j->c.tau, 1));
  ok = ok && soft(lcbp_free_energy(j->scratch, &Fs));
  ok = ok && soft(lcbp_step(j->lat, (int)j->k)) && soft(lcbp_free_energy(j->lat, &Fp));
  if (ok) {
    gF = std::fabs(Fs - Fp) / std::fabs(Fp);
    ok = soft(q_gap(j, &gQ));
  }
  if (soft.hard) return soft.hard;
  j->st.segments += 1;
  j->st.last_gap_F = gF;
  j->st.last_gap_Q = gQ;
  if (std::isfinite(gF) && std::isfinite(gQ)) {
    j->st.judged += 1;
    j->st.mean_gap_F += (gF - j->st.mean_gap_F) / (double)j->st.judged;
    j->st.mean_gap_Q += (gQ - j->st.mean_gap_Q) / (double)j->st.judged;
  }
  const bool pass = ok && std::isfinite(gF) && gF <= j->c.tol_F &&
                    (j->c.tol_Q <= 0.0 || (std::isfinite(gQ) && gQ <= j->c.tol_Q));
  const long long seg = calls * j->k;
  if (pass) {
    j->st.accepted += 1;
    j->st.surrogate_calls += calls;
    j->st.plain_steps += j->k;
    if (gF > j->st.max_gap_F) j->st.max_gap_F = gF;
    const long long te = t + seg + j->k;
    if (log_every > 0 && te % log_every == 0) {
      double F = 0, D = 0;
      rc = measure(j, thr, &F, &D);
      if (rc) return rc;
      j->pt.push_back(te);
      j->pF.push_back(F);
      j->pD.push_back(D);
    }
    *accepted = true;
    return LCBP_OK;
  }
  // roll back and redo the segment with plain steps
  j->st.fallbacks += 1;
  j->pt.clear();
  j->pF.clear();
  j->pD.clear();
  rc = lcbp_restore(j->lat, j->snap);
  if (!rc) rc = plain(j, t, seg, log_every, thr, j->pt, j->pF, j->pD);
  *accepted = false;
  return rc;
}

}  // namespace

extern "C" {

int lcbp_judge_create(lcbp_lattice* h, lcbp_surrogate* s, const lcbp_judge_config* c, lcbp_judge** out) {
  if (!out) return fail(LCBP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!h || !s || !c) return fail(LCBP_EINVAL, "lattice, surrogate and config must not be NULL");
  if (c->calls_per_segment < 1) return fail(LCBP_EINVAL, "calls_per_segment must be >= 1");
  if (!std::isfinite(c->kappa) || !std::isfinite(c->tau) || !(c->tol_F >= 0.0) || !std::isfinite(c->tol_Q) ||
      c->warmup_steps < 0)
    return fail(LCBP_EINVAL, "need finite kappa, tau, tol_Q, tol_F >= 0 and warmup_steps >= 0");
  int k = 0;
  int rc0 = lcbp_surrogate_get_steps(s, &k);
  if (rc0) return rc0;
  auto* j = new lcbp_judge();
  j->k = k;
  j->lat = h;
  j->sur = s;
  j->c = *c;
  int rc = lattice_clone(h, &j->scratch);
  const size_t bytes = lcbp_snapshot_bytes(h);
  cudaError_t e = cudaSuccess;
  if (!rc) e = cudaMalloc(&j->snap, bytes);
  if (!rc && e == cudaSuccess) e = cudaMalloc(&j->snap2, bytes);
  if (!rc && e == cudaSuccess) e = cudaMalloc(&j->red, state_check_scratch_bytes() + 8);
  if (!rc && e == cudaSuccess) e = cudaMallocHost(&j->h_red, sizeof(double));
  if (!rc && e != cudaSuccess) {
    cudaGetLastError();
    rc = fail(LCBP_ENOMEM, "judge buffers of 2 x %zu bytes", bytes);
  }
  if (rc) {
    lcbp_judge_destroy(j);
    return rc;
  }
  j->st.last_gap_F = j->st.last_gap_Q = NAN;
  *out = j;
  return LCBP_OK;
}

int lcbp_judge_destroy(lcbp_judge* j) {
  if (!j) return LCBP_OK;
  if (j->scratch) lcbp_destroy(j->scratch);
  if (j->snap) cudaFree(j->snap);
  if (j->snap2) cudaFree(j->snap2);
  if (j->red) cudaFree(j->red);
  if (j->h_red) cudaFreeHost(j->h_red);
  delete j;
  return LCBP_OK;
}

int lcbp_judge_advance(lcbp_judge* j, long long t_end, int log_every, double defect_threshold, long long* log_t,
                       double* log_F, double* log_defect, int capacity, int* nlog) {
  if (!j) return fail(LCBP_EINVAL, "null judge handle");
  if (nlog) *nlog = 0;
  if (log_every < 0 || log_every % j->k != 0)
    return fail(LCBP_EINVAL, "log_every must be a multiple of %lld (or 0)", j->k);
  long long t = j->st.t;
  if (t_end < t) return fail(LCBP_EINVAL, "t_end %lld is before the run's time %lld", t_end, t);
  if (log_every > 0) {
    if (t_end % j->k != 0)
      return fail(LCBP_EINVAL, "with logging, t_end must be a multiple of %lld", j->k);
    if (!log_t || !log_F || !log_defect || !nlog) return fail(LCBP_EINVAL, "log arrays and nlog must not be NULL");
    const long long marks = t_end / log_every - t / log_every;
    if (marks > capacity) return fail(LCBP_EINVAL, "%lld log entries do not fit capacity %d", marks, capacity);
  }
  int written = 0;
  auto commit = [&]() {
    for (size_t k = 0; k < j->pt.size(); ++k) {
      log_t[written] = j->pt[k];
      log_F[written] = j->pF[k];
      log_defect[written] = j->pD[k];
      ++written;
    }
    if (nlog) *nlog = written;
  };
  while (t < t_end) {
    // a segment that stands also takes the judge's k plain steps: it must fit before t_end
    const int calls = (int)std::min<long long>(j->c.calls_per_segment, (t_end - t) / j->k - 1);
    int rc;
    long long adv;
    if (t < j->c.warmup_steps) {  // the plain warm-up (to a multiple of k, so segments stay aligned)
      j->pt.clear();
      j->pF.clear();
      j->pD.clear();
      const long long w = (j->c.warmup_steps + j->k - 1) / j->k * j->k;
      adv = std::min(w, t_end) - t;
      rc = plain(j, t, adv, log_every, defect_threshold, j->pt, j->pF, j->pD);
    } else if (calls < 1) {  // fewer than 2k steps left: plain
      j->pt.clear();
      j->pF.clear();
      j->pD.clear();
      adv = t_end - t;
      rc = plain(j, t, adv, log_every, defect_threshold, j->pt, j->pF, j->pD);
    } else {
      bool accepted = false;
      rc = segment(j, t, calls, log_every, defect_threshold, &accepted);
      adv = calls * j->k + (accepted ? j->k : 0);
    }
    if (rc) return rc;
    commit();
    t += adv;
    j->st.t = t;
  }
  return LCBP_OK;
}

int lcbp_judge_get_stats(lcbp_judge* j, lcbp_judge_stats* out) {
  if (!j || !out) return fail(LCBP_EINVAL, "judge and out must not be NULL");
  *out = j->st;
  return LCBP_OK;
}

}  // extern "C"
