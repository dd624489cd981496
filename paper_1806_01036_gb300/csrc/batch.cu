// batch.cu — many independent blocks of uneven n and k orthogonalized by one
// CUDA graph launch, with launch shapes picked by an autotuner.
//
// The paper's solvers orthogonalize one block at a time (Sec. 4.2); a
// process that serves many of them (a batch of subspace iterations, or the
// blocks of one iteration spread over independent problems) would otherwise
// pay one host round of launches per block and leave the GPU idle while a
// small block's k-by-k eigensolve runs in one CTA.  Here:
//
//   * every block runs the sequence of a single eo_svqb / eo_cholqr call
//     (ctx.cuh: enqueue_orth) on its own device workspace, with a launch
//     shape that depends on its own (k, n) only, so its result does not
//     depend on the batch it is in (with the default shapes it is bitwise
//     that of the single call);
//   * the blocks are spread over B branches (longest first, each to the
//     least-loaded branch) and captured once into a CUDA graph whose branches
//     run concurrently: one eo_batch_run is one cudaGraphLaunch;
//   * the streaming kernels of a block are capped at a number of CTAs chosen
//     per (k, n bucket, mode) by the autotuner, so that small blocks take a
//     few SMs and run side by side instead of spreading thinly over all 152.
//
// Autotuner: for a key (k, floor(log2 n), mode) it times the block's Gram
// and update kernels on a synthetic n x k buffer (n = 2^(bucket + 1/2)) for a
// coarse set of CTA caps, then refines around the best, and keeps the cap
// with the least SM time (CTAs x duration) -- the quantity a batch that fills
// the GPU with concurrent blocks spends -- preferring more CTAs within 5 %.
// Results live in the context and, when eo_tune_cache names a file, on disk
// (one line per key, tagged with the device name).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <vector>

#include "ctx.cuh"

struct eo_batch {
  eo_ctx* ctx = nullptr;
  int nb = 0;
  size_t slot_bytes = 0;
  int branches = 0;
  uint64_t nodes = 0;  // kernels per run
  void* mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<eo::Tile> tiles;
};

namespace eo {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kTuneMinBucket = 12;  // below 4096 rows the launch shape hardly matters: defaults
constexpr int kTuneReps = 3;

int n_bucket(int64_t n) {
  int b = 0;
  while (b < 62 && (2ll << b) <= n) ++b;
  return b;
}

// Deterministic values in [-1, 1) with varied exponents (splitmix64 of the index).
__global__ void tune_fill_kernel(double* x, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    const double m = (double)(z >> 11) * 0x1p-53 * 2.0 - 1.0;
    x[i] = ldexp(m, -(int)((z >> 3) & 7));
  }
}

// Identity transform (hi = I, lo = 0) for the timed updates.
__global__ void tune_identity_kernel(SmallWs* ws) {
  for (int t = threadIdx.x; t < KMAX * KMAX; t += blockDim.x) {
    ws->Zh[t] = (t % KMAX) == (t / KMAX) ? 1.0 : 0.0;
    ws->Zl[t] = 0.0;
  }
}

struct Candidate {
  int cap, ctas;
  float ms;
};

// Picks the cap with the least CTAs x time, preferring more CTAs within 5 %.
int pick(const std::vector<Candidate>& c) {
  double best = 1e300;
  for (const Candidate& x : c) best = std::min(best, (double)x.ctas * x.ms);
  int cap = 0, ctas = -1;
  for (const Candidate& x : c)
    if ((double)x.ctas * x.ms <= 1.05 * best && x.ctas > ctas) {
      ctas = x.ctas;
      cap = x.cap;
    }
  return cap;
}

class Tuner {
 public:
  explicit Tuner(eo_ctx* ctx) : ctx_(ctx) {}
  ~Tuner() {
    if (s_) cudaStreamSynchronize(s_);
    if (buf_) cudaFree(buf_);
    if (e0_) cudaEventDestroy(e0_);
    if (e1_) cudaEventDestroy(e1_);
    if (s_) cudaStreamDestroy(s_);
  }

  // Sizes the buffers for the largest key; returns a CUDA error, if any.
  cudaError_t prepare(int64_t n_max, int k_max) {
    cudaError_t e = cudaStreamCreateWithFlags(&s_, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0_);
    if (e == cudaSuccess) e = cudaEventCreate(&e1_);
    if (e != cudaSuccess) return e;
    elems_ = (size_t)n_max * k_max;
    parts_bytes_ = align_up(std::max<size_t>(
        {dd_gram_scratch(n_max, k_max, k_max, true), fx_update_tmp_bytes(n_max, k_max), kAlign}));
    const size_t bytes = align_up(elems_ * sizeof(double)) + parts_bytes_ + align_up(sizeof(SmallWs)) +
                         align_up(2 * sizeof(double) * KMAX * KMAX);
    e = cudaMalloc(&buf_, bytes);
    if (e != cudaSuccess) {
      buf_ = nullptr;
      return e;
    }
    x_ = static_cast<double*>(buf_);
    parts_ = static_cast<char*>(buf_) + align_up(elems_ * sizeof(double));
    ws_ = reinterpret_cast<SmallWs*>(static_cast<char*>(parts_) + parts_bytes_);
    g_ = reinterpret_cast<double*>(reinterpret_cast<char*>(ws_) + align_up(sizeof(SmallWs)));
    tune_fill_kernel<<<1024, 256, 0, s_>>>(x_, elems_);
    tune_identity_kernel<<<1, 256, 0, s_>>>(ws_);
    return cudaGetLastError();
  }

  // Tile of a key, timed on n = 2^(bucket + 1/2) rows.
  cudaError_t tune(int k, int bucket, Tile* out) {
    // a multiple of 16 rows keeps every column 16-byte aligned (the tensor-core
    // Gram engine reads through TMA and needs that)
    const int64_t n = std::min<int64_t>((int64_t)std::ldexp(1.4142135623730951, bucket), elems_ / k) / 16 * 16;
    cudaError_t e;
    auto gram = [&](int cap) {
      return launch_dd_gram(n, k, x_, n, k, x_, n, true, parts_, g_, g_ + KMAX * KMAX, KMAX, nullptr, s_, cap);
    };
    auto update = [&](int cap) {
      return launch_fx_update(n, k, x_, n, ws_->Zh, ws_->Zl, false, nullptr, s_, cap, parts_, parts_bytes_);
    };
    int gcap = 0, rcap = 0;
    e = search([&](int cap) { return dd_gram_ctas(n, k, k, true, cap); }, gram, &gcap);
    if (e != cudaSuccess) return e;
    e = search([&](int cap) { return fx_update_ctas(n, k, cap); }, update, &rcap);
    if (e != cudaSuccess) return e;
    out->gram = gcap;
    out->row = rcap;
    return cudaSuccess;
  }

 private:
  template <class Ctas, class Launch>
  cudaError_t search(Ctas ctas_of, Launch launch, int* best_cap) {
    std::vector<Candidate> seen;
    auto try_cap = [&](int cap) -> cudaError_t {
      cap = std::max(1, std::min(152, cap));
      const int c = ctas_of(cap);
      for (const Candidate& x : seen)
        if (x.ctas == c) return cudaSuccess;  // same launch shape as a cap already timed
      cudaError_t e = launch(cap);  // warm-up
      if (e != cudaSuccess) return e;
      float t[kTuneReps];
      for (int r = 0; r < kTuneReps; ++r) {
        e = cudaEventRecord(e0_, s_);
        if (e == cudaSuccess) e = launch(cap);
        if (e == cudaSuccess) e = cudaEventRecord(e1_, s_);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1_);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t[r], e0_, e1_);
        if (e != cudaSuccess) return e;
      }
      std::sort(t, t + kTuneReps);
      seen.push_back(Candidate{cap, c, t[kTuneReps / 2]});
      return cudaSuccess;
    };
    for (int cap : {4, 8, 16, 38, 76, 152}) {  // coarse
      cudaError_t e = try_cap(cap);
      if (e != cudaSuccess) return e;
    }
    const int mid = pick(seen);
    for (int cap : {mid * 2 / 3, mid * 3 / 4, mid * 4 / 3, mid * 3 / 2}) {  // fine, around the best
      cudaError_t e = try_cap(cap);
      if (e != cudaSuccess) return e;
    }
    *best_cap = pick(seen);
    return cudaSuccess;
  }

  eo_ctx* ctx_;
  cudaStream_t s_ = nullptr;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
  void* buf_ = nullptr;
  double* x_ = nullptr;
  double* g_ = nullptr;
  void* parts_ = nullptr;
  SmallWs* ws_ = nullptr;
  size_t elems_ = 0, parts_bytes_ = 0;
};

std::string device_tag(int device) {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string s = p.name;
  for (char& c : s)
    if (c == ' ') c = '_';
  return s + "/" + std::to_string(p.multiProcessorCount);
}

// Cache lines: "k bucket prec gram_cap row_cap device_tag".
void load_cache(eo_ctx* ctx) {
  std::ifstream in(ctx->tune_path);
  if (!in) return;
  const std::string tag = device_tag(ctx->device);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ls(line);
    TuneKey k{};
    Tile t{};
    std::string dev;
    if (!(ls >> k.k >> k.bucket >> k.prec >> t.gram >> t.row >> dev)) continue;
    if (dev == tag) ctx->tuned[k] = t;
  }
}

bool save_cache(eo_ctx* ctx) {
  if (ctx->tune_path.empty()) return true;
  const std::string tag = device_tag(ctx->device);
  std::vector<std::string> keep;  // other devices' lines
  {
    std::ifstream in(ctx->tune_path);
    std::string line;
    while (in && std::getline(in, line)) {
      std::istringstream ls(line);
      int a, b, c, d, e;
      std::string dev;
      if ((ls >> a >> b >> c >> d >> e >> dev) && dev != tag) keep.push_back(line);
    }
  }
  const std::string tmp = ctx->tune_path + ".tmp";
  {
    std::ofstream out(tmp, std::ios::trunc);
    if (!out) return false;
    for (const std::string& l : keep) out << l << "\n";
    for (const auto& kv : ctx->tuned)
      out << kv.first.k << " " << kv.first.bucket << " " << kv.first.prec << " " << kv.second.gram << " "
          << kv.second.row << " " << tag << "\n";
    if (!out) return false;
  }
  return std::rename(tmp.c_str(), ctx->tune_path.c_str()) == 0;
}

struct Slot {  // per-block device workspace
  DevStatus st;
  SmallWs ws;
};

void free_batch(eo_batch* bt) {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->mem) cudaFree(bt->mem);
  delete bt;
}

// A batch under construction: released unless handed out.
struct Owned {
  eo_batch* p;
  explicit Owned(eo_batch* b) : p(b) {}
  ~Owned() { free_batch(p); }
  eo_batch* operator->() { return p; }
  eo_batch* release() {
    eo_batch* b = p;
    p = nullptr;
    return b;
  }
};

// Streams and events of one fork/join capture; an unfinished capture is
// ended and its graph dropped on the way out.
struct Capture {
  int B;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> ev;
  bool capturing = false;
  explicit Capture(int b) : B(b), br(b, nullptr), ev(b + 1, nullptr) {}
  cudaError_t create() {
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int s = 0; s < B && e == cudaSuccess; ++s) e = cudaStreamCreateWithFlags(&br[s], cudaStreamNonBlocking);
    for (int s = 0; s <= B && e == cudaSuccess; ++s) e = cudaEventCreateWithFlags(&ev[s], cudaEventDisableTiming);
    return e;
  }
  cudaError_t begin() {
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) capturing = true;
    return e;
  }
  // every branch waits for what the capture stream has so far
  cudaError_t fork() {
    cudaError_t e = cudaEventRecord(ev[B], cap);
    for (int s = 0; s < B && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(br[s], ev[B], 0);
    return e;
  }
  // the capture stream waits for every branch
  cudaError_t join() {
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < B && e == cudaSuccess; ++s) {
      e = cudaEventRecord(ev[s], br[s]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[s], 0);
    }
    return e;
  }
  cudaError_t end(cudaGraph_t* g) {
    cudaError_t e = join();
    if (e != cudaSuccess) return e;
    capturing = false;
    return cudaStreamEndCapture(cap, g);
  }
  ~Capture() {
    if (capturing) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(cap, &junk);
      if (junk) cudaGraphDestroy(junk);
      cudaGetLastError();
    }
    for (cudaStream_t s : br)
      if (s) cudaStreamDestroy(s);
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    if (cap) cudaStreamDestroy(cap);
  }
};

}  // namespace
}  // namespace eo

using namespace eo;

extern "C" {

eo_status eo_tune_cache(eo_ctx* ctx, const char* path) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  ctx->tune_path = path ? path : "";
  if (!ctx->tune_path.empty()) load_cache(ctx);
  return EO_OK;
}

eo_status eo_batch_create(eo_ctx* ctx, int nblocks, const eo_block* blocks, eo_batch_method method, double tol,
                          int passes, eo_prec prec, int* out_dev, int branches, int flags, eo_batch** out) {
  if (!ctx) return EO_EINVAL;
  ctx->err.clear();
  EO_CHECK(out != nullptr, EO_EINVAL, "eo_batch_create: null output handle%s", "");
  *out = nullptr;
  EO_CHECK(nblocks >= 1 && blocks != nullptr, EO_EINVAL, "eo_batch_create: no blocks%s", "");
  EO_CHECK(method == EO_BATCH_SVQB || method == EO_BATCH_CHOLQR, EO_EINVAL, "eo_batch_create: bad method%s %lld", "",
           (long long)method);
  EO_CHECK(valid_prec(prec), EO_EINVAL, "eo_batch_create: bad precision mode%s %lld", "", (long long)prec);
  EO_CHECK(passes >= 0 && passes <= 2, EO_EINVAL, "eo_batch_create: passes must be 0, 1 or 2%s", "");
  EO_CHECK(branches >= 0 && branches <= 64, EO_EINVAL, "eo_batch_create: branches must be in [0, 64]%s", "");
  for (int b = 0; b < nblocks; ++b) {
    const eo_block& x = blocks[b];
    EO_CHECK(x.n >= 0 && x.k >= 1 && x.k <= KMAX, EO_EINVAL, "eo_batch_create: bad sizes of block %s%lld", "",
             (long long)b);
    EO_CHECK(x.X != nullptr || x.n == 0, EO_EINVAL, "eo_batch_create: null X in block %s%lld", "", (long long)b);
    EO_CHECK(x.ldx >= std::max<int64_t>(1, x.n), EO_EINVAL, "eo_batch_create: ldx too small in block %s%lld", "",
             (long long)b);
    EO_CHECK(!(x.Z_hi || x.Z_lo) || x.ldz >= x.k, EO_EINVAL, "eo_batch_create: ldz too small in block %s%lld", "",
             (long long)b);
  }
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_batch_create: cannot select device%s", "");

  // launch shapes: tuned per (k, n bucket) for the compensated mode
  std::vector<Tile> tiles(nblocks);
  if (prec == EO_DD && !(flags & EO_BATCH_NO_TUNE)) {
    std::vector<TuneKey> missing;
    int64_t n_max = 0;
    int k_max = 0;
    for (int b = 0; b < nblocks; ++b) {
      const int bk = n_bucket(blocks[b].n);
      if (blocks[b].n < (1ll << kTuneMinBucket)) continue;
      const TuneKey key{blocks[b].k, bk, (int)prec};
      if (ctx->tuned.count(key) || std::find_if(missing.begin(), missing.end(), [&](const TuneKey& m) {
                                     return !(m < key) && !(key < m);
                                   }) != missing.end())
        continue;
      missing.push_back(key);
      n_max = std::max<int64_t>(n_max, (int64_t)std::ldexp(1.4142135623730951, bk) + 1);
      k_max = std::max(k_max, key.k);
    }
    if (!missing.empty()) {
      Tuner t(ctx);
      cudaError_t e = t.prepare(n_max, k_max);
      if (e != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (autotuner buffers)", e);
      for (const TuneKey& key : missing) {
        Tile tl;
        e = t.tune(key.k, key.bucket, &tl);
        if (e != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (autotuner)", e);
        ctx->tuned[key] = tl;
      }
      if (!save_cache(ctx)) return fail(ctx, EO_EINVAL, "eo_batch_create: cannot write the tuning cache %s",
                                        ctx->tune_path.c_str());
    }
    for (int b = 0; b < nblocks; ++b) {
      if (blocks[b].n < (1ll << kTuneMinBucket)) continue;
      tiles[b] = ctx->tuned[TuneKey{blocks[b].k, n_bucket(blocks[b].n), (int)prec}];
    }
  }

  // branches: longest block first, each to the least-loaded branch
  const int B = std::max(1, std::min(nblocks, branches > 0 ? branches : 16));
  std::vector<int> order(nblocks), branch_of(nblocks);
  for (int b = 0; b < nblocks; ++b) order[b] = b;
  auto cost = [&](int b) { return (double)blocks[b].n * (blocks[b].k + 4) + 2e4 * blocks[b].k * blocks[b].k; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<double> load(B, 0.0);
  for (int b : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch_of[b] = s;
    load[s] += cost(b);
  }

  // device memory: one workspace per block, one partial-sum area per
  // branch, the job list of the batched factorizations
  size_t parts = kAlign;
  for (int b = 0; b < nblocks; ++b) parts = std::max(parts, orth_scratch(blocks[b].n, blocks[b].k, prec));
  parts = align_up(parts);
  const size_t slot = align_up(sizeof(Slot));
  const size_t jobs_bytes = align_up(sizeof(SmallJob) * nblocks);
  Owned bt(new eo_batch());
  bt->ctx = ctx;
  bt->nb = nblocks;
  bt->branches = B;
  bt->tiles = tiles;
  bt->slot_bytes = slot;
  const size_t total = slot * nblocks + parts * B + jobs_bytes;
  cudaError_t e = cudaMalloc(&bt->mem, total);
  if (e != cudaSuccess) {
    bt->mem = nullptr;
    cudaGetLastError();
    return fail(ctx, EO_ENOMEM, "eo_batch_create: cannot allocate %s%lld bytes", "", (long long)total);
  }
  char* base = static_cast<char*>(bt->mem);
  auto slot_of = [&](int b) { return reinterpret_cast<Slot*>(base + slot * b); };  // pitch slot_bytes
  char* parts0 = base + slot * nblocks;
  SmallJob* jobs_dev = reinterpret_cast<SmallJob*>(parts0 + parts * B);
  const Mode small_mode = pipe_mode(prec) == MODE_DD ? MODE_DD : MODE_FP64;
  std::vector<SmallJob> jobs(nblocks);
  int kmax = 1;
  for (int b = 0; b < nblocks; ++b) {
    const eo_block& x = blocks[b];
    jobs[b] = SmallJob{x.k, &slot_of(b)->ws, &slot_of(b)->st, x.Z_hi, x.Z_lo, x.ldz,
                       tol < 0 ? svqb_default_tol(small_mode, x.k) : tol, out_dev ? out_dev + b : nullptr};
    kmax = std::max(kmax, x.k);
  }
  // longest first: CTAs start in index order, so the widest factorizations
  // take SMs of their own and the short ones fill in around them
  std::stable_sort(jobs.begin(), jobs.end(), [](const SmallJob& a, const SmallJob& b) { return a.k > b.k; });
  if ((e = cudaMemcpy(jobs_dev, jobs.data(), sizeof(SmallJob) * nblocks, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(ctx, "eo_batch_create (job list)", e);

  // capture: fork from a private stream onto B branch streams, join back
  Capture c(B);
  if ((e = c.create()) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (streams)", e);
  if ((e = c.begin()) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (begin capture)", e);
  uint64_t nodes = 0;
  const bool chol = method == EO_BATCH_CHOLQR;
  auto args_of = [&](int b) {
    const eo_block& x = blocks[b];
    return OrthArgs{chol, x.n, x.k, x.X, x.ldx, nullptr, nullptr, 0, x.Z_hi, x.Z_lo, x.ldz, tol, passes, prec,
                    out_dev ? out_dev + b : nullptr};
  };
  auto res_of = [&](int b) {
    const int s = branch_of[b];
    OrthRes r{&slot_of(b)->st, &slot_of(b)->ws, parts0 + parts * s, c.br[s], tiles[b]};
    r.parts_bytes = parts;
    return r;
  };
  if (flags & EO_BATCH_CHAINS) {
    // each block's whole sequence on its branch
    if ((e = c.fork()) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (fork)", e);
    for (int b : order) {
      const char* where = "";
      if ((e = enqueue_orth(args_of(b), res_of(b), &nodes, &where)) != cudaSuccess)
        return cuda_fail(ctx, (std::string("eo_batch_create (") + where + ")").c_str(), e);
    }
  } else {
    // by phase: the Gram matrices of a pass on the branches, all k-by-k
    // factorizations of the pass in one launch (one CTA per block, every
    // SM), then the updates on the branches
    if ((e = launch_status_init_batched(jobs_dev, nblocks, c.cap)) != cudaSuccess)
      return cuda_fail(ctx, "eo_batch_create (status init)", e);
    if ((e = c.fork()) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (fork)", e);
    const int npass = passes == 1 ? 1 : 2;
    for (int p = 0; p < npass; ++p) {
      for (int b : order)
        if ((e = enqueue_orth_step(args_of(b), res_of(b), p, OrthStep::kGram, &nodes)) != cudaSuccess)
          return cuda_fail(ctx, "eo_batch_create (Gram)", e);
      if ((e = c.join()) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (join)", e);
      if ((e = launch_small_batched(chol, small_mode, nblocks, kmax, jobs_dev, p, passes, c.cap)) != cudaSuccess)
        return cuda_fail(ctx, "eo_batch_create (factorizations)", e);
      if ((e = c.fork()) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (fork)", e);
      for (int b : order)
        if ((e = enqueue_orth_step(args_of(b), res_of(b), p, OrthStep::kUpdate, &nodes)) != cudaSuccess)
          return cuda_fail(ctx, "eo_batch_create (update)", e);
    }
  }
  if ((e = c.end(&bt->graph)) != cudaSuccess) return cuda_fail(ctx, "eo_batch_create (end capture)", e);
  if ((e = cudaGraphInstantiate(&bt->exec, bt->graph, 0)) != cudaSuccess) {
    bt->exec = nullptr;
    return cuda_fail(ctx, "eo_batch_create (instantiate)", e);
  }
  size_t count = 0;  // kernel nodes actually captured (a call with nothing to do launches nothing)
  if ((e = cudaGraphGetNodes(bt->graph, nullptr, &count)) != cudaSuccess)
    return cuda_fail(ctx, "eo_batch_create (graph nodes)", e);
  bt->nodes = count;
  (void)nodes;
  *out = bt.release();
  return EO_OK;
}

eo_status eo_batch_run(eo_batch* bt) {
  if (!bt || !bt->ctx) return EO_EINVAL;
  eo_ctx* ctx = bt->ctx;
  ctx->err.clear();
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "eo_batch_run: cannot select device%s", "");
  EO_CUDA(cudaGraphLaunch(bt->exec, ctx->stream), "eo_batch_run");
  ctx->launches += bt->nodes;
  return EO_OK;
}

eo_status eo_batch_destroy(eo_batch* bt) {
  if (!bt) return EO_EINVAL;
  DeviceGuard g(bt->ctx->device);
  cudaStreamSynchronize(bt->ctx->stream);  // a launched graph may still be running
  free_batch(bt);
  return EO_OK;
}

eo_status eo_batch_tile(const eo_batch* bt, int block, int* gram_ctas, int* row_ctas) {
  if (!bt || block < 0 || block >= bt->nb) return EO_EINVAL;
  if (gram_ctas) *gram_ctas = bt->tiles[block].gram;
  if (row_ctas) *row_ctas = bt->tiles[block].row;
  return EO_OK;
}

// One int of every block's status (at byte offset `off` of DevStatus) into host memory.
static eo_status copy_status_field(eo_batch* bt, size_t off, int* host, const char* name) {
  if (!bt || !host) return EO_EINVAL;
  eo_ctx* ctx = bt->ctx;
  ctx->err.clear();
  DeviceGuard g(ctx->device);
  EO_CHECK(g.ok, EO_ECUDA, "%s: cannot select device", name);
  EO_CUDA(cudaStreamSynchronize(ctx->stream), name);
  const char* src = static_cast<const char*>(bt->mem) + offsetof(Slot, st) + off;
  EO_CUDA(cudaMemcpy2D(host, sizeof(int), src, bt->slot_bytes, sizeof(int), bt->nb, cudaMemcpyDeviceToHost), name);
  return EO_OK;
}

eo_status eo_batch_passes(eo_batch* bt, int* passes_host) {
  // gate[2] of a block's status enables its second pass
  eo_status s = copy_status_field(bt, offsetof(DevStatus, gate) + 2 * sizeof(int), passes_host, "eo_batch_passes");
  if (s != EO_OK) return s;
  for (int b = 0; b < bt->nb; ++b) passes_host[b] = passes_host[b] ? 2 : 1;
  return EO_OK;
}

eo_status eo_batch_sweeps(eo_batch* bt, int* sweeps_host) {
  return copy_status_field(bt, offsetof(DevStatus, sweeps), sweeps_host, "eo_batch_sweeps");
}

int64_t eo_batch_kernels(const eo_batch* bt) { return bt ? (int64_t)bt->nodes : -1; }

int eo_batch_branches(const eo_batch* bt) { return bt ? bt->branches : -1; }

}  // extern "C"
