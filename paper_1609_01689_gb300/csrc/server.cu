// Serving: many LOBPCG solves advanced together (continuous batching).
//
// Default: the lockstep engine (lockstep.cu) -- one iteration of every admitted solve per progress
// call, each kernel one launch for all solves. The stream engines below run each admitted solve as
// a resumable task (lobpcg.cu) on its own stream. One progress pass steps
// each task until it waits on the device (an event it recorded) or asks for H times a block.
// The products asked for in the same pass go out as one batched launch per arithmetic class on
// the server's stream: the server stream waits on each task's "ready" event, launches, and each
// task stream waits on the batch's "done" event, so no host synchronisation sits between a
// task's work and the shared SpMM. Admission is by a device-memory budget (matrix + solver
// state per solve) and a slot count; any queued request that fits is admitted, in arrival order.
#include <string.h>

#include <chrono>
#include <deque>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

constexpr int RING = 8;  // job-table buffers in flight

size_t matrix_bytes(const lob_matrix* m) {
  const lob_tiles& T = m->T;
  size_t b = (size_t)T.nnz * 4;  // (r, c)
  if (T.v64) b += (size_t)T.nnz * 8;
  if (T.v32) b += (size_t)T.nnz * 4;
  if (T.v32lo) b += (size_t)T.nnz * 4;
  if (T.rv) b += (size_t)T.nnz * 8;
  if (T.cperm) b += (size_t)(T.nnz + 8) * 2;
  if (T.rvp) b += (size_t)(T.nnz + 8) * 10;  // the parity-ordered copies (rvp, cpermp)
  b += (size_t)(T.nt + 1) * 8 + (size_t)T.ntiles * 8 + (size_t)(T.ntiles + 1) * 12;
  b += (size_t)T.nchunks * 2 * (LOB_TILE + 1) * 2;
  if (m->P.Q) b += (size_t)m->P.nblk * m->P.bp * m->P.bp * 4 + (size_t)m->P.nblk * m->P.bp * 4;
  b += (size_t)T.nt * LOB_TILE * 16 * 8;  // staged X at the widest batched class
  return b;
}

struct Req {
  int64_t id = 0;
  lob_request r{};
  lob_task* t = nullptr;
  lob_ltask* lt = nullptr;  // lockstep engine
  cudaStream_t st = nullptr;
  cudaEvent_t ready = nullptr;
  size_t bytes = 0;
  bool wait_sync = false, want = false, finished = false;
  lob_result res{};
};

}  // namespace

struct lob_server {
  lob_server_opts o{};
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::deque<Req*> queue;
  std::vector<Req*> active;
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_id = 1;
  size_t used = 0;
  cudaStream_t sst = nullptr;
  std::vector<cudaStream_t> spool;
  std::vector<cudaEvent_t> epool;
  lob_spmm_job* jh = nullptr;  // pinned [RING][jcap]
  lob_spmm_job* jd = nullptr;  // device [RING][jcap]
  cudaEvent_t jev[RING] = {};
  bool jev_used[RING] = {};
  int ring = 0;
  cudaEvent_t batch_done = nullptr;
  lob_engine* E = nullptr;  // lockstep engine (engine == LOB_ENGINE_LOCKSTEP)
  lob_server_stats stats{};

  double now() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  int get_stream(cudaStream_t* s) {
    if (!spool.empty()) { *s = spool.back(); spool.pop_back(); return LOB_OK; }
    LOB_CUDA(cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
    return LOB_OK;
  }
  int get_event(cudaEvent_t* e) {
    if (!epool.empty()) { *e = epool.back(); epool.pop_back(); return LOB_OK; }
    LOB_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return LOB_OK;
  }

  void retire(Req* q, int rc) {
    if (q->lt) {
      double lam[64];
      rc = lob_engine_result(E, q->lt, lam, &q->res.stats, nullptr);
      if (rc == LOB_OK || rc == LOB_ERR_NOCONV) memcpy(q->res.lambda, lam, q->r.k * sizeof(double));
      q->lt = nullptr;
    }
    if (q->t) {
      if (rc == LOB_OK || rc == LOB_ERR_NOCONV || rc > 0) {
        double lam[64];
        rc = lob_task_result(q->t, lam, &q->res.stats);
        // a persistent SpMM kernel of this solve that gave up on a bounded wait voids the result
        if (lob_matrix_fault_take(q->r.H, q->st) != 0) rc = LOB_ERR_CUDA;
        if (rc == LOB_OK || rc == LOB_ERR_NOCONV) memcpy(q->res.lambda, lam, q->r.k * sizeof(double));
      }
      lob_task_destroy(q->t);  // stream-ordered release of the solver state
      q->t = nullptr;
    }
    if (q->st) { spool.push_back(q->st); q->st = nullptr; }
    if (q->ready) { epool.push_back(q->ready); q->ready = nullptr; }
    used -= q->bytes;
    q->res.rc = rc;
    q->res.state = LOB_REQ_DONE;
    q->res.t_done_ms = now();
    q->finished = true;
    stats.finished++;
  }

  int admit() {
    for (auto it = queue.begin(); it != queue.end();) {
      if ((int)active.size() >= o.max_active) break;
      Req* q = *it;
      if (used + q->bytes > o.budget_bytes) { ++it; continue; }
      if (E) {
        const bool guess = q->r.opts.n_small >= 3 * q->r.nb && q->r.opts.n_small < q->r.H->T.n;
        if (lob_engine_free_slots(E) < (guess ? 2 : 1)) break;
        it = queue.erase(it);
        used += q->bytes;
        if (used > stats.bytes_peak) stats.bytes_peak = used;
        q->res.state = LOB_REQ_RUNNING;
        q->res.t_admit_ms = now();
        stats.admitted++;
        active.push_back(q);
        const lob_matrix* H = q->r.H;
        int rc = lob_ensure_xs(H, (size_t)H->T.nt * LOB_TILE * 16 * 8);
        if (rc == LOB_OK)
          rc = lob_engine_add(E, q->r.H, q->r.k, q->r.nb, q->r.tol, &q->r.opts, q->r.X, H->T.n, q->id, &q->lt);
        if (rc != LOB_OK) { q->lt = nullptr; retire(q, rc); }
        continue;
      }
      it = queue.erase(it);
      used += q->bytes;
      if (used > stats.bytes_peak) stats.bytes_peak = used;
      q->res.state = LOB_REQ_RUNNING;
      q->res.t_admit_ms = now();
      stats.admitted++;
      active.push_back(q);
      int rc = get_stream(&q->st);
      if (rc == LOB_OK) rc = get_event(&q->ready);
      const lob_matrix* H = q->r.H;
      if (rc == LOB_OK) rc = lob_ensure_xs(H, (size_t)H->T.nt * LOB_TILE * 16 * 8);
      if (rc == LOB_OK) {
        lob_solve_opts so = q->r.opts;
        so.stream = q->st;
        rc = lob_task_create(q->r.H, q->r.k, q->r.nb, q->r.tol, nullptr, &so, q->r.X, H->T.n, q->st, false, &q->t);
      }
      if (rc != LOB_OK) retire(q, rc);
    }
    return LOB_OK;
  }

  // Step q until it waits on the device, asks for an SpMM or finishes. Returns steps taken.
  int advance(Req* q, std::vector<Req*>& want) {
    int moved = 0;
    while (!q->finished) {
      lob_task* leaf = lob_task_leaf(q->t);
      if (q->wait_sync) {
        const cudaError_t e = cudaEventQuery(lob_task_event(leaf));
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) { cudaGetLastError(); retire(q, LOB_ERR_CUDA); break; }
        q->wait_sync = false;
      }
      if (q->want) break;
      const int r = lob_task_step(q->t);
      moved++;
      if (r < 0) { retire(q, r); break; }
      if (r == LOB_TASK_SYNC) { q->wait_sync = true; continue; }
      if (r == LOB_TASK_SPMM) { q->want = true; want.push_back(q); break; }
      retire(q, LOB_OK);
    }
    return moved;
  }

  int launch(std::vector<Req*>& want) {
    const int nj = (int)want.size();
    if (o.engine == LOB_ENGINE_STREAMS) {  // one launch per solve, on the solve's own stream
      for (Req* q : want) {
        const int rc = lob_task_spmm_direct(lob_task_leaf(q->t));
        if (rc != LOB_OK) retire(q, rc);
        stats.spmm_launches++;
      }
      stats.spmm_products += nj;
      return LOB_OK;
    }
    const int slot = ring;
    ring = (ring + 1) % RING;
    if (jev_used[slot]) LOB_CUDA(cudaEventSynchronize(jev[slot]));  // its job table was consumed
    std::vector<const lob_matrix*> ms(nj);
    std::vector<const double*> X(nj);
    std::vector<double*> Y(nj);
    std::vector<int> ncol(nj), mode(nj);
    std::vector<int64_t> nact(nj);
    for (int j = 0; j < nj; j++) {
      Req* q = want[j];
      lob_task_spmm_args(lob_task_leaf(q->t), &ms[j], &X[j], &Y[j], &ncol[j], &mode[j], &nact[j]);
      LOB_CUDA(cudaEventRecord(q->ready, q->st));
      LOB_CUDA(cudaStreamWaitEvent(sst, q->ready, 0));
    }
    int nk = 0;
    const int rc = lob_spmm_batch_launch(ms.data(), X.data(), Y.data(), ncol.data(), mode.data(), nact.data(), nj,
                                         jh + (size_t)slot * o.max_active, jd + (size_t)slot * o.max_active, sst,
                                         &nk);
    LOB_CUDA(cudaEventRecord(jev[slot], sst));
    jev_used[slot] = true;
    LOB_CUDA(cudaEventRecord(batch_done, sst));
    for (Req* q : want) {
      if (rc != LOB_OK) { retire(q, rc); continue; }
      LOB_CUDA(cudaStreamWaitEvent(q->st, batch_done, 0));
    }
    stats.spmm_launches += nk;
    stats.spmm_products += nj;
    return LOB_OK;
  }

  int progress_lockstep(int* n_done) {
    const int64_t fin0 = stats.finished;
    LOB_TRY(admit());
    if (lob_engine_ntasks(E) > 0) {
      std::vector<lob_ltask*> done;
      LOB_TRY(lob_engine_round(E, done));
      for (lob_ltask* t : done) {
        // find the request of this solve (its tag is the request id)
        int64_t id = 0;
        for (Req* q : active)
          if (q->lt == t) { id = q->id; retire(q, LOB_OK); break; }
        (void)id;
      }
      size_t w = 0;
      for (size_t i = 0; i < active.size(); i++)
        if (!active[i]->finished) active[w++] = active[i];
      active.resize(w);
      stats.spmm_launches = lob_engine_spmm_launches(E);
      stats.spmm_products = lob_engine_spmm_products(E);
    }
    if (stats.finished > fin0) LOB_TRY(admit());
    if (n_done) *n_done = (int)(stats.finished - fin0);
    return LOB_OK;
  }

  int progress(int wait, int* n_done) {
    LOB_CUDA(cudaSetDevice(device));
    stats.progress_calls++;
    if (E) return progress_lockstep(n_done);
    const int64_t fin0 = stats.finished;
    LOB_TRY(admit());
    int moved = 0;
    std::vector<Req*> want;
    for (size_t i = 0; i < active.size(); i++) moved += advance(active[i], want);
    while (!want.empty()) {
      LOB_TRY(launch(want));
      std::vector<Req*> again;
      for (Req* q : want) {
        q->want = false;
        if (!q->finished) moved += advance(q, again);
      }
      want.swap(again);
    }
    // retire finished solves from the active set
    size_t w = 0;
    for (size_t i = 0; i < active.size(); i++)
      if (!active[i]->finished) active[w++] = active[i];
    active.resize(w);
    if (stats.finished > fin0) LOB_TRY(admit());
    if (wait && moved == 0 && stats.finished == fin0) {
      for (Req* q : active)
        if (q->wait_sync) {
          LOB_CUDA(cudaEventSynchronize(lob_task_event(lob_task_leaf(q->t))));
          break;
        }
    }
    if (n_done) *n_done = (int)(stats.finished - fin0);
    return LOB_OK;
  }
};

extern "C" {

int lob_spmm_batch(int32_t njobs, lob_matrix* const* H, const double* const* X, double* const* Y, const int32_t* nb,
                   const int32_t* mode, const int64_t* n_act, void* stream) {
  if (njobs < 0 || (njobs > 0 && (!H || !X || !Y || !nb || !mode))) return LOB_ERR_ARG;
  if (njobs == 0) return LOB_OK;
  for (int j = 0; j < njobs; j++)
    if (!H[j] || !X[j] || !Y[j]) return LOB_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<const lob_matrix*> ms(H, H + njobs);
  std::vector<int> ncol(nb, nb + njobs), md(mode, mode + njobs);
  for (int j = 0; j < njobs; j++) {
    if (ncol[j] < 1 || ncol[j] > 16) return LOB_ERR_ARG;
    const lob_matrix* m = ms[j];
    LOB_TRY(lob_ensure_xs(m, (size_t)m->T.nt * LOB_TILE * 16 * 8));
  }
  lob_spmm_job* jh = nullptr;
  lob_spmm_job* jd = nullptr;
  if (cudaHostAlloc((void**)&jh, njobs * sizeof(lob_spmm_job), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return LOB_ERR_NOMEM;
  }
  if (cudaMallocAsync((void**)&jd, njobs * sizeof(lob_spmm_job), st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(jh);
    return LOB_ERR_NOMEM;
  }
  int rc = lob_spmm_batch_launch(ms.data(), X, Y, ncol.data(), md.data(), n_act, njobs, jh, jd, st);
  cudaFreeAsync(jd, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == LOB_OK) rc = LOB_ERR_CUDA;
  cudaFreeHost(jh);
  return rc;
}

int lob_server_create(const lob_server_opts* o, lob_server** out) {
  if (!out) return LOB_ERR_ARG;
  *out = nullptr;
  lob_server* s = new lob_server();
  if (o) s->o = *o;
  if (s->o.budget_bytes == 0) s->o.budget_bytes = 60ull << 30;
  if (s->o.max_active <= 0) s->o.max_active = 64;
  if (s->o.engine < LOB_ENGINE_LOCKSTEP || s->o.engine > LOB_ENGINE_STREAMS) {
    delete s;
    return LOB_ERR_ARG;
  }
  s->t0 = std::chrono::steady_clock::now();
  int rc = LOB_OK;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->sst, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->batch_done, cudaEventDisableTiming) != cudaSuccess)
    rc = LOB_ERR_CUDA;
  for (int i = 0; rc == LOB_OK && i < RING; i++)
    if (cudaEventCreateWithFlags(&s->jev[i], cudaEventDisableTiming) != cudaSuccess) rc = LOB_ERR_CUDA;
  if (rc == LOB_OK && s->o.engine == LOB_ENGINE_LOCKSTEP) rc = lob_engine_create(2 * s->o.max_active, s->sst, &s->E);
  const size_t jb = (size_t)RING * s->o.max_active * sizeof(lob_spmm_job);
  if (rc == LOB_OK && (cudaHostAlloc((void**)&s->jh, jb, cudaHostAllocDefault) != cudaSuccess ||
                       cudaMalloc((void**)&s->jd, jb) != cudaSuccess))
    rc = LOB_ERR_NOMEM;
  if (rc != LOB_OK) {
    cudaGetLastError();
    lob_server_destroy(s);
    return rc;
  }
  *out = s;
  return LOB_OK;
}

int lob_server_submit(lob_server* s, const lob_request* r, int64_t* id) {
  if (!s || !r || !id || !r->H) return LOB_ERR_ARG;
  const lob_matrix* H = r->H;
  const lob_solve_opts& o = r->opts;
  if (r->k < 1 || r->nb < r->k || r->nb > 16 || !(r->tol > 0.0) || H->T.n < 3 * r->nb) return LOB_ERR_ARG;
  if (o.mode != LOB_MODE_FP64 && o.mode != LOB_MODE_MIXED) return LOB_ERR_ARG;
  if (o.mode == LOB_MODE_MIXED && (!H->T.v32 || !H->T.v64)) return LOB_ERR_ARG;
  if (o.mode == LOB_MODE_FP64 && !H->T.v64) return LOB_ERR_ARG;
  if (o.precond && !((H->P.bp >= 1 && H->P.bp <= 64) || H->P.bp == LOB_TILE)) return LOB_ERR_ARG;
  if (o.precond_solve < LOB_PSOLVE_FOM || o.precond_solve > LOB_PSOLVE_ABS || o.precond_steps < 0 ||
      o.precond_steps > 3)
    return LOB_ERR_ARG;
  // the diagonal tiles are solved by Krylov steps only (nothing is factorised for a direct solve)
  if (o.precond && H->P.bp == LOB_TILE && o.precond_solve != LOB_PSOLVE_FOM && o.precond_solve != LOB_PSOLVE_MINRES)
    return LOB_ERR_ARG;
  if (o.rr_arith < LOB_ARITH_FP64 || o.rr_arith > LOB_ARITH_DF || o.refine_arith < LOB_ARITH_FP64 ||
      o.refine_arith > LOB_ARITH_DF)
    return LOB_ERR_ARG;
  Req* q = new Req();
  q->id = s->next_id++;
  q->r = *r;
  q->bytes = matrix_bytes(H) + (s->E ? lob_engine_task_bytes(H, r->nb, o.n_small) : lob_task_bytes(H, r->nb, o.n_small));
  if (q->bytes > s->o.budget_bytes) { delete q; return LOB_ERR_ARG; }
  q->res.state = LOB_REQ_QUEUED;
  q->res.bytes = q->bytes;
  q->res.t_submit_ms = s->now();
  s->queue.push_back(q);
  s->reqs[q->id] = q;
  s->stats.submitted++;
  *id = q->id;
  return LOB_OK;
}

int lob_server_progress(lob_server* s, int32_t wait, int32_t* n_done) {
  if (!s) return LOB_ERR_ARG;
  int nd = 0;
  const int rc = s->progress(wait, &nd);
  if (n_done) *n_done = nd;
  return rc;
}

int lob_server_poll(lob_server* s, int64_t id, lob_result* out) {
  if (!s || !out) return LOB_ERR_ARG;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return LOB_ERR_ARG;
  Req* q = it->second;
  *out = q->res;
  if (q->res.state == LOB_REQ_DONE) {
    s->reqs.erase(it);
    delete q;
  }
  return LOB_OK;
}

int lob_server_stats_get(const lob_server* s, lob_server_stats* out) {
  if (!s || !out) return LOB_ERR_ARG;
  *out = s->stats;
  out->active = (int64_t)s->active.size();
  out->queued = (int64_t)s->queue.size();
  out->bytes_in_use = s->used;
  if (s->E) {
    long long r = 0;
    lob_engine_times(s->E, &out->host_ms, &out->wait_ms, &r);
    out->rounds = r;
  }
  return LOB_OK;
}

int lob_server_destroy(lob_server* s) {
  if (!s) return LOB_ERR_ARG;
  cudaSetDevice(s->device);
  for (Req* q : s->active)
    if (q->st) cudaStreamSynchronize(q->st);
  if (s->sst) cudaStreamSynchronize(s->sst);
  if (s->E) { lob_engine_destroy(s->E); s->E = nullptr; }
  for (Req* q : s->active) {
    if (q->t) lob_task_destroy(q->t);
    if (q->st) cudaStreamSynchronize(q->st), cudaStreamDestroy(q->st);
    if (q->ready) cudaEventDestroy(q->ready);
  }
  for (auto& kv : s->reqs) delete kv.second;
  for (cudaStream_t x : s->spool) cudaStreamSynchronize(x), cudaStreamDestroy(x);
  for (cudaEvent_t e : s->epool) cudaEventDestroy(e);
  for (int i = 0; i < RING; i++)
    if (s->jev[i]) cudaEventDestroy(s->jev[i]);
  if (s->batch_done) cudaEventDestroy(s->batch_done);
  if (s->sst) cudaStreamDestroy(s->sst);
  if (s->jh) cudaFreeHost(s->jh);
  if (s->jd) cudaFree(s->jd);
  delete s;
  return LOB_OK;
}

}  // extern "C"
