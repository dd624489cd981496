// serve.cu — a request server for many concurrent eigensolves: each keeps its
// basis V resident on the device and submits blocks Y to orthogonalize
// against it (phase I: Y - V (V^T Y), phase II: compensated CholQR of the
// result; arXiv:1806.01036, Sec. 4.2).
//
// Runtime:
//   * a server thread admits queued requests (admission.h: FIFO, one request
//     at a time per basis, device-memory budget) onto slots -- a stream, a
//     context with its scratch reserved up front, and the k-by-k Gram buffer --
//     as soon as a slot and the memory are free (continuous batching: requests
//     that arrive while others run join as they can; their kernels overlap on
//     the GPU);
//   * each admitted request is enqueued on its slot's stream with the
//     library's own calls (eo_project with the fused Gram, eo_cholqr with the
//     automatic second pass) followed by a host callback that stamps its
//     completion; the server thread then frees its slot and memory;
//   * latency = completion stamp - submission time (host steady clock).
// Every slot runs the default launch shapes, and compensated sums are exact,
// so a request's result is bitwise the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "admission.h"
#include "ctx.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Basis {
  int64_t n;
  int kv;
  const double* V;
  int64_t ldv;
};

struct Request;

struct Slot {
  eo_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  double* M = nullptr;  // Gram matrix of the projected block: hi then lo, EO_KMAX x EO_KMAX each
  int64_t req = -1;
};

}  // namespace

struct eo_server {
  eo_ctx* parent = nullptr;
  int device = 0;
  eo::Admission adm;
  std::vector<Slot> slots;
  std::vector<Basis> bases;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  int64_t next_id = 0;
  std::unordered_map<int64_t, Request*> reqs;
  std::vector<int64_t> completed;  // done or failed, not yet reported by eo_server_poll
  size_t max_parts = 0;            // scratch reserved in every slot
  eo_server(size_t budget, int nslots) : adm(budget, nslots) {}
};

namespace {

struct Request {
  eo_server* srv;
  int64_t id;
  int basis, k;
  const double* Y;
  int64_t ldy;
  double* Yout;
  int64_t ldyo;
  double *R_hi, *R_lo;
  int ldr;
  int* info_dev;
  size_t bytes;
  double t_submit = 0, t_start = 0, t_done = 0;
  int status = 0;  // 0 queued, 1 running, 2 done, 3 failed
  int slot = -1;
  std::atomic<bool> gpu_done{false};
};

void CUDART_CB on_done(void* p) {
  Request* r = static_cast<Request*>(p);
  r->t_done = now_s();
  r->gpu_done.store(true, std::memory_order_release);
  r->srv->cv.notify_all();
}

// Enqueues request r on slot s (lock held).  Returns false on a CUDA error.
bool start(eo_server* srv, Slot& s, Request& r) {
  const Basis& b = srv->bases[r.basis];
  const int K = EO_KMAX;
  double* mh = s.M;
  double* ml = s.M + K * K;
  eo_status st = eo_project(s.ctx, b.n, b.kv, b.V, b.ldv, r.k, r.Y, r.ldy, r.Yout, r.ldyo, nullptr, nullptr, 0, mh,
                            ml, K, EO_DD);
  if (st == EO_OK)
    st = eo_cholqr(s.ctx, b.n, r.k, r.Yout, r.ldyo, mh, ml, K, r.R_hi, r.R_lo, r.ldr, 0, EO_DD, r.info_dev);
  if (st != EO_OK) return false;
  return cudaLaunchHostFunc(s.stream, on_done, &r) == cudaSuccess;
}

void serve_loop(eo_server* srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    // reap what the GPU has finished
    for (Slot& s : srv->slots) {
      if (s.req < 0) continue;
      Request* r = srv->reqs[s.req];
      if (!r->gpu_done.load(std::memory_order_acquire)) continue;
      r->status = 2;
      srv->adm.finish(r->id, r->basis);
      srv->completed.push_back(r->id);
      s.req = -1;
    }
    // admit what fits
    for (const eo::AdmitItem& it : srv->adm.admit()) {
      Request* r = srv->reqs[it.id];
      int si = 0;
      while (srv->slots[si].req >= 0) ++si;  // admit() never hands out more than the free slots
      Slot& s = srv->slots[si];
      r->slot = si;
      r->t_start = now_s();
      r->status = 1;
      s.req = r->id;
      if (!start(srv, s, *r)) {
        cudaGetLastError();
        r->status = 3;
        srv->adm.finish(r->id, r->basis);
        srv->completed.push_back(r->id);
        s.req = -1;
      }
    }
    srv->cv.notify_all();  // waiters in eo_server_wait
    srv->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

}  // namespace

using namespace eo;

extern "C" {

eo_status eo_server_create(eo_ctx* ctx, size_t hbm_budget, int slots, eo_server** out) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(out != nullptr, EO_EINVAL, "eo_server_create: null output handle%s", "");
  *out = nullptr;
  EO_CHECK(slots >= 1 && slots <= 256, EO_EINVAL, "eo_server_create: slots must be in [1, 256]%s", "");
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_server_create: cannot select device%s", "");
  eo_server* srv = new eo_server(hbm_budget, slots);
  srv->parent = ctx;
  srv->device = ctx->device;
  srv->slots.resize(slots);
  const size_t mbytes = 2 * sizeof(double) * EO_KMAX * EO_KMAX;
  eo_status st = EO_OK;
  for (Slot& s : srv->slots) {
    if ((st = eo_create(&s.ctx, ctx->device)) != EO_OK) break;
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&s.M, mbytes) != cudaSuccess) {
      cudaGetLastError();
      st = EO_ENOMEM;
      break;
    }
    eo_set_stream(s.ctx, s.stream);
  }
  if (st == EO_OK && !srv->adm.add_resident(mbytes * slots)) st = EO_ENOMEM;
  if (st != EO_OK) {
    for (Slot& s : srv->slots) {  // the context first: it synchronizes the slot's stream
      if (s.ctx) eo_destroy(s.ctx);
      if (s.M) cudaFree(s.M);
      if (s.stream) cudaStreamDestroy(s.stream);
    }
    delete srv;
    return fail(ctx, st, "eo_server_create: cannot set up the slots%s", "");
  }
  srv->th = std::thread(serve_loop, srv);
  *out = srv;
  return EO_OK;
}

eo_status eo_server_destroy(eo_server* srv) {
  if (!srv) return EO_EINVAL;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  if (srv->th.joinable()) srv->th.join();
  DeviceGuard g(srv->device);
  for (Slot& s : srv->slots) {  // the context first: it synchronizes the slot's stream
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.ctx) eo_destroy(s.ctx);
    if (s.M) cudaFree(s.M);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  for (auto& kv : srv->reqs) delete kv.second;
  delete srv;
  return EO_OK;
}

eo_status eo_server_add_basis(eo_server* srv, int64_t n, int kv, const double* V, int64_t ldv, int* basis_id) {
  if (!srv) return EO_EINVAL;
  eo_ctx* ctx = srv->parent;
  EO_CHECK(n >= 0 && kv >= 1 && kv <= KMAX && basis_id, EO_EINVAL, "eo_server_add_basis: bad sizes%s", "");
  EO_CHECK(V != nullptr || n == 0, EO_EINVAL, "eo_server_add_basis: null V%s", "");
  EO_CHECK(ldv >= std::max<int64_t>(1, n), EO_EINVAL, "eo_server_add_basis: ldv too small%s", "");
  DeviceGuard g(srv->device);
  std::lock_guard<std::mutex> lk(srv->mu);
  const size_t bytes = (size_t)n * kv * sizeof(double);
  if (!srv->adm.add_resident(bytes))
    return fail(ctx, EO_ENOMEM, "eo_server_add_basis: %s%lld bytes do not fit the budget", "", (long long)bytes);
  // every slot reserves the scratch of the largest request this basis can get (k <= EO_KMAX)
  const size_t need = std::max(dd_gram_scratch(n, kv, KMAX, false), dd_gram_scratch(n, KMAX, KMAX, true));
  if (need > srv->max_parts) {
    for (Slot& s : srv->slots) {
      eo_status st = reserve_scratch(s.ctx, need);
      if (st != EO_OK) return fail(ctx, st, "eo_server_add_basis: cannot reserve slot scratch%s", "");
    }
    srv->max_parts = need;
  }
  srv->bases.push_back(Basis{n, kv, V, ldv});
  *basis_id = (int)srv->bases.size() - 1;
  return EO_OK;
}

eo_status eo_server_submit(eo_server* srv, int basis_id, int k, const double* Y, int64_t ldy, double* Yout,
                           int64_t ldyo, double* R_hi, double* R_lo, int ldr, int* info_dev, int64_t* req_id) {
  if (!srv) return EO_EINVAL;
  eo_ctx* ctx = srv->parent;
  std::lock_guard<std::mutex> lk(srv->mu);
  EO_CHECK(basis_id >= 0 && basis_id < (int)srv->bases.size() && req_id, EO_EINVAL,
           "eo_server_submit: bad basis%s %lld", "", (long long)basis_id);
  const Basis& b = srv->bases[basis_id];
  const int64_t mn = std::max<int64_t>(1, b.n);
  EO_CHECK(k >= 1 && k <= KMAX && ldy >= mn && ldyo >= mn, EO_EINVAL, "eo_server_submit: bad sizes%s", "");
  EO_CHECK((Y && Yout) || b.n == 0, EO_EINVAL, "eo_server_submit: null block%s", "");
  EO_CHECK(!(R_hi || R_lo) || ldr >= k, EO_EINVAL, "eo_server_submit: ldr too small%s", "");
  const size_t bytes = (size_t)b.n * k * sizeof(double) * (Yout == Y ? 1 : 2);
  if (!srv->adm.can_ever_fit(bytes))
    return fail(ctx, EO_ENOMEM, "eo_server_submit: the block (%s%lld bytes) can never fit the budget", "",
                (long long)bytes);
  Request* r = new Request();
  r->srv = srv;
  r->id = srv->next_id++;
  r->basis = basis_id;
  r->k = k;
  r->Y = Y;
  r->ldy = ldy;
  r->Yout = Yout;
  r->ldyo = ldyo;
  r->R_hi = R_hi;
  r->R_lo = R_lo;
  r->ldr = ldr;
  r->info_dev = info_dev;
  r->bytes = bytes;
  r->t_submit = now_s();
  srv->reqs[r->id] = r;
  srv->adm.push(AdmitItem{r->id, basis_id, bytes});
  *req_id = r->id;
  srv->cv.notify_all();
  return EO_OK;
}

eo_status eo_server_wait(eo_server* srv, int64_t req_id, double timeout_s, int* status, double* latency_ms) {
  if (!srv) return EO_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(req_id);
  if (it == srv->reqs.end()) return EO_EINVAL;
  Request* r = it->second;
  const double t_end = now_s() + timeout_s;
  while (r->status < 2) {
    if (now_s() > t_end) return EO_ETIMEOUT;
    srv->cv.wait_for(lk, std::chrono::microseconds(500));
  }
  if (status) *status = r->status == 2 ? EO_OK : EO_ECUDA;
  if (latency_ms) *latency_ms = 1e3 * (r->t_done - r->t_submit);
  return EO_OK;
}

eo_status eo_server_poll(eo_server* srv, int max_out, int64_t* ids, double* latency_ms, double* queue_ms,
                         int* statuses, int* n_out) {
  if (!srv || !n_out || max_out < 0) return EO_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  int n = 0;
  while (n < max_out && !srv->completed.empty()) {
    const int64_t id = srv->completed.front();
    srv->completed.erase(srv->completed.begin());
    Request* r = srv->reqs[id];
    if (ids) ids[n] = id;
    if (latency_ms) latency_ms[n] = r->status == 2 ? 1e3 * (r->t_done - r->t_submit) : -1.0;
    if (queue_ms) queue_ms[n] = 1e3 * (r->t_start - r->t_submit);
    if (statuses) statuses[n] = r->status == 2 ? EO_OK : EO_ECUDA;
    ++n;
  }
  *n_out = n;
  return EO_OK;
}

eo_status eo_server_stats(eo_server* srv, size_t* resident, size_t* peak_inflight, int* peak_running, int* queued,
                          int* running, uint64_t* kernels) {
  if (!srv) return EO_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (kernels) {
    uint64_t n = 0;
    for (const Slot& s : srv->slots) n += eo_kernel_launches(s.ctx);
    *kernels = n;
  }
  if (resident) *resident = srv->adm.resident();
  if (peak_inflight) *peak_inflight = srv->adm.peak_inflight();
  if (peak_running) *peak_running = (int)srv->adm.peak_running();
  if (queued) *queued = (int)srv->adm.queued();
  if (running) *running = (int)srv->adm.running();
  return EO_OK;
}

// The admission policy alone, driven by a discrete-event simulation (no GPU):
// request i arrives at arrival[i] on basis[i], holds bytes[i] and runs for
// duration[i] once admitted; start[i] receives its admission time (-1 if it
// can never fit).  resident_bytes are reserved first.  Returns the peak number
// of requests running at once (or -1 on bad arguments).
EO_API int eo_admission_simulate(size_t budget, int slots, size_t resident_bytes, int nreq, const int* basis,
                          const int64_t* bytes, const double* arrival, const double* duration, double* start) {
  if (slots < 1 || nreq < 0 || (nreq > 0 && (!basis || !bytes || !arrival || !duration || !start))) return -1;
  Admission adm(budget, slots);
  if (!adm.add_resident(resident_bytes)) return -1;
  std::vector<int> order(nreq);
  for (int i = 0; i < nreq; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return arrival[a] < arrival[b]; });
  std::vector<std::pair<double, int>> running;  // (finish time, request)
  int next = 0, peak = 0;
  for (int i = 0; i < nreq; ++i) start[i] = -1.0;
  double t = 0.0;
  while (next < nreq || !running.empty()) {
    // next event: an arrival or a completion, completions first at equal times
    double t_arr = next < nreq ? arrival[order[next]] : 1e300;
    double t_fin = 1e300;
    int fin = -1;
    for (int j = 0; j < (int)running.size(); ++j)
      if (running[j].first < t_fin) {
        t_fin = running[j].first;
        fin = j;
      }
    if (fin >= 0 && t_fin <= t_arr) {
      t = t_fin;
      const int id = running[fin].second;
      adm.finish(id, basis[id]);
      running.erase(running.begin() + fin);
    } else {
      t = t_arr;
      const int id = order[next++];
      if (!adm.can_ever_fit((size_t)bytes[id])) continue;
      adm.push(AdmitItem{id, basis[id], (size_t)bytes[id]});
    }
    for (const AdmitItem& it : adm.admit()) {
      start[it.id] = t;
      running.emplace_back(t + duration[it.id], (int)it.id);
    }
    peak = std::max(peak, (int)running.size());
  }
  return peak;
}

}  // extern "C"
