// Serving: a request loop with continuous batching over the expansion and alignment kernels.
//
// Requests (template id, B host volumes, S starts) are queued by bh_serve_submit.  One worker thread
// owns all device work: it retires finished batches (event query), then admits waiting requests --
// merging the head request with later ones of the same box edge and start count -- as long as a stream
// slot is free and the batch's device footprint fits the remaining HBM budget.
// A batch is: stream-ordered allocation from the server's own memory pool (which keeps up to the budget
// mapped, so steady-state allocations never go back to the driver), host->device copies, expansion
// (bh::expand_into with the batch's own scratch, so batches on different streams never share scratch),
// one bh_align_batch launch with a per-subtomogram template index, device->host copies into pinned
// staging, stream-ordered free, event.  Up to max_inflight bulk batches are on the device at once.
//
// Optionally (express_slots > 0) two classes: a request whose estimated device time (a throughput model
// of the expansion and the marching ascent) is at most express_ms is "express" and runs on one of
// express_slots streams created at the device's highest priority, so the block scheduler gives its
// kernels the next free SM slots ahead of bulk work already queued; bulk requests use the max_inflight
// low-priority streams.  Within a class admission keeps arrival order (the head of a class is never
// overtaken by a later request of the same class); an express request may take a free bulk stream
// when no bulk request waits.  Off by default: under bursts of large requests the measured p99 latency
// of the mixed Poisson workload was lower with one class.
//
// A request larger than `piece` subtomograms is admitted piece by piece: its first piece is queued at
// submission, and each time a piece is admitted the next one joins the END of the queue, behind requests
// that arrived in the meantime, so a burst of large requests no longer holds every stream slot while
// small ones wait.  Pieces draw the random starts their subtomograms would draw unsplit, so a result does
// not depend on the split; the request completes with its last piece.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "bh_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxTemplatesPerBox = 64;
constexpr int kScratchRows = 512;  // expansion pass of a batch (rows of the 128-row M tile)

struct Box {
  int N = 0;
  bh_plan* plan = nullptr;
  float* d_tmpl = nullptr;  // [kMaxTemplatesPerBox][Nb] complex
  int n_tmpl = 0;
  int stages[3];
  int nstages = 0;
};

struct Template {
  int N;
  int row;
};

struct Req {
  uint64_t ticket;
  bh_request r;
  int N;
  int row;
  bool express = false;
  Clock::time_point t_submit, t_done;
  int status = BH_PENDING;
  // a request admitted in pieces: each piece points at its request; the request counts what is left
  std::shared_ptr<Req> parent;
  int pieces_left = 0;  // pieces not finished yet
  int next_off = 0;     // first subtomogram not yet queued as a piece
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* h_starts = nullptr;  // pinned staging
  int* h_tidx = nullptr;
  const float** h_vptr = nullptr;  // volume addresses (in-place ingestion)
  float* h_quat = nullptr;
  float* h_score = nullptr;
  size_t cap_starts = 0, cap_b = 0;
  bool busy = false;
  std::vector<std::shared_ptr<Req>> reqs;
  size_t bytes = 0;
  int launch_status = BH_OK;
  bool express = false;  // high-priority stream reserved for express batches
};

// Device bytes of a batch: its volumes (unless read in place from the request buffers, then a table of
// B addresses), coefficients, starts, template indices, results and expansion scratch (the 8 parity-class
// projections of each row over the fundamental voxels, and the real GEMM output).
size_t batch_bytes(const bh_plan* p, int B, int S, bool in_place) {
  const size_t rows = (size_t)bh::round_up(std::min(B, kScratchRows), bh::kGemmBM);
  const size_t vols = in_place ? (size_t)B * sizeof(void*) : (size_t)B * p->N * p->N * p->N * 4;
  return vols + (size_t)B * p->Nb * 8 + (size_t)B * S * 16 + (size_t)B * 4 + (size_t)B * 20 +
         rows * ((size_t)8 * p->VF_pad * 4 + (size_t)p->Nb_pad * 4) + 4 * 256;
}

// Work of one evaluation of Eq. 2 with its gradient at band L (flop): 30 per orbit-step of the
// d-recursion and 46 per orbit.
double eval_flop(int L) {
  double steps = 0.0;
  for (int m = 0; m <= L; ++m) steps += (2.0 * m + 1.0) * (L - m + 1);
  const double orbits = (L + 1.0) * (L + 1.0);
  return 30.0 * (steps - orbits) + 46.0 * orbits;
}

// Estimated device time (ms) of a batch of B subtomograms: the expansion at 1 PFLOP/s of executed tensor
// work (three BF16 products) or 40 TFLOP/s (FP32), but no less than one pass of the basis table over HBM
// (every batch streams it once: 1.8 GB for the folded BF16 hi/lo table at 64^3) at 6.5 TB/s; the ascent at
// 20 TFLOP/s of FP32 work.  Throughputs measured for these kernels; used only to classify requests.
double est_ms(const bh_plan* p, const int* stages, int nstages, int steps, int B, int S) {
  const double gemm = 2.0 * p->VF_pad * p->Nb_pad;  // the folded GEMM: fundamental voxels x padded table rows
  const double expand = (p->mode == BH_MODE_BF16_SPLIT) ? 3.0 * gemm / 1e12 : gemm / 40e12;
  const double table = 4.0 * p->Nb_pad * p->VF_pad / 6.5e12;  // FP32, or BF16 hi + lo: 4 bytes per entry
  double align = 0.0;
  for (int i = 0; i < nstages; ++i) align += eval_flop(stages[i]);
  align *= (double)S * (1.0 + steps) / 20e12;
  return 1e3 * (std::max(B * expand, table) + B * align);
}

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct bh_server {
  int device = 0;
  bh_serve_opts o{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
  std::map<int, Box> boxes;
  std::vector<Template> templates;
  std::vector<Slot> slots;
  cudaMemPool_t pool = nullptr;
  double express_ms = 0.0;
  bool in_place = false;  // the device reads request volumes in host memory coherently (no H2D copy)
  uint64_t next_ticket = 1;
  size_t used = 0;
  bool stop = false, paused = false;
  uint64_t submitted = 0, completed = 0, batches = 0, express_batches = 0, in_place_batches = 0;
  std::atomic<uint64_t> staging_allocs{0};
  double launch_ms_total = 0.0, launch_ms_max = 0.0;  // worker time spent enqueueing batches
  std::thread worker;
  std::mutex plan_mu;  // serialises plan creation / template upload with the worker's launches
};

namespace {

// Pinned staging of a slot for B subtomograms with S starts.  Sized at server creation for max_batch
// subtomograms and up to kStagedStarts starts, so that the batch path never frees pinned memory (a
// pinned free waits for the whole device); only a request with more starts grows it.
constexpr int kStagedStarts = 64;

int grow_staging(bh_server* s, Slot& sl, int B, int S) {
  if (sl.cap_b < (size_t)B) {
    cudaFreeHost(sl.h_tidx);
    cudaFreeHost(sl.h_quat);
    cudaFreeHost(sl.h_score);
    cudaFreeHost(sl.h_vptr);
    sl.h_tidx = nullptr;
    sl.h_quat = sl.h_score = nullptr;
    sl.h_vptr = nullptr;
    sl.cap_b = 0;
    BH_CUDA_TRY(cudaMallocHost(&sl.h_vptr, (size_t)B * sizeof(float*)));
    BH_CUDA_TRY(cudaMallocHost(&sl.h_tidx, (size_t)B * sizeof(int)));
    BH_CUDA_TRY(cudaMallocHost(&sl.h_quat, (size_t)B * 4 * sizeof(float)));
    BH_CUDA_TRY(cudaMallocHost(&sl.h_score, (size_t)B * sizeof(float)));
    sl.cap_b = (size_t)B;
    ++s->staging_allocs;
  }
  if (sl.cap_starts < (size_t)B * S * 4) {
    cudaFreeHost(sl.h_starts);
    sl.h_starts = nullptr;
    sl.cap_starts = 0;
    BH_CUDA_TRY(cudaMallocHost(&sl.h_starts, (size_t)B * S * 4 * sizeof(float)));
    sl.cap_starts = (size_t)B * S * 4;
    ++s->staging_allocs;
  }
  return BH_OK;
}

int launch_batch(bh_server* s, Slot& sl, int N, int S) {
  const bh::Range range_("bh_serve batch");
  Box& box = s->boxes[N];
  bh_plan* p = box.plan;
  int B = 0;
  for (auto& r : sl.reqs) B += r->r.B;
  {
    const int rc = grow_staging(s, sl, std::max(B, s->o.max_batch), S);
    if (rc != BH_OK) return rc;
  }
  int off = 0;
  for (auto& r : sl.reqs) {
    const bh_request& q = r->r;
    if (q.starts) {
      std::memcpy(sl.h_starts + (size_t)off * S * 4, q.starts, sizeof(float) * (size_t)q.B * S * 4);
    } else {
      bh_random_starts(q.seed, q.B, S, sl.h_starts + (size_t)off * S * 4);
    }
    for (int b = 0; b < q.B; ++b) sl.h_tidx[off + b] = r->row;
    off += q.B;
  }
  cudaStream_t st = sl.stream;
  const size_t N3 = (size_t)N * N * N;
  const int rows = bh::round_up(std::min(B, kScratchRows), bh::kGemmBM);
  const bool in_place = s->in_place;
  float *d_vols = nullptr, *d_coef = nullptr, *d_starts = nullptr, *d_quat = nullptr, *d_score = nullptr;
  float *d_sx = nullptr, *d_sc = nullptr;
  const float** d_vptr = nullptr;
  int* d_tidx = nullptr;
  cudaMemPool_t pool = s->pool;
  if (in_place)
    BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_vptr, (size_t)B * sizeof(float*), pool, st));
  else
    BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_vols, (size_t)B * N3 * 4, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_coef, (size_t)B * p->Nb * 8, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_starts, (size_t)B * S * 16, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_tidx, (size_t)B * 4, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_quat, (size_t)B * 16, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_score, (size_t)B * 4, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_sx, (size_t)rows * 8 * p->VF_pad * 4, pool, st));
  BH_CUDA_TRY(cudaMallocFromPoolAsync((void**)&d_sc, (size_t)rows * p->Nb_pad * 4, pool, st));
  off = 0;
  for (auto& r : sl.reqs) {
    if (in_place) {
      for (int b = 0; b < r->r.B; ++b) sl.h_vptr[off + b] = r->r.vols + (size_t)b * N3;
    } else {
      BH_CUDA_TRY(cudaMemcpyAsync(d_vols + (size_t)off * N3, r->r.vols, sizeof(float) * (size_t)r->r.B * N3,
                                  cudaMemcpyHostToDevice, st));
    }
    off += r->r.B;
  }
  if (in_place) BH_CUDA_TRY(cudaMemcpyAsync(d_vptr, sl.h_vptr, (size_t)B * sizeof(float*), cudaMemcpyHostToDevice, st));
  BH_CUDA_TRY(cudaMemcpyAsync(d_starts, sl.h_starts, (size_t)B * S * 16, cudaMemcpyHostToDevice, st));
  BH_CUDA_TRY(cudaMemcpyAsync(d_tidx, sl.h_tidx, (size_t)B * 4, cudaMemcpyHostToDevice, st));
  int rc = bh::expand_into(p, d_vols, d_vptr, B, d_coef, d_sx, d_sc, rows, st);
  if (rc == BH_OK) {
    bh_align_opts ao{};
    ao.tmpl_index = d_tidx;
    ao.n_templates = box.n_tmpl;
    ao.newton = s->o.newton;
    rc = bh_align_batch(p, box.d_tmpl, d_coef, B, d_starts, S, box.stages, box.nstages, s->o.steps, d_quat, d_score,
                        &ao, st);
  }
  if (rc == BH_OK) {
    BH_CUDA_TRY(cudaMemcpyAsync(sl.h_quat, d_quat, (size_t)B * 16, cudaMemcpyDeviceToHost, st));
    BH_CUDA_TRY(cudaMemcpyAsync(sl.h_score, d_score, (size_t)B * 4, cudaMemcpyDeviceToHost, st));
  }
  for (void* ptr : {(void*)d_vols, (void*)d_vptr, (void*)d_coef, (void*)d_starts, (void*)d_tidx, (void*)d_quat,
                    (void*)d_score, (void*)d_sx, (void*)d_sc})
    if (ptr) cudaFreeAsync(ptr, st);
  BH_CUDA_TRY(cudaEventRecord(sl.done, st));
  return rc;
}

void retire(bh_server* s, Slot& sl, int status) {
  // caller holds s->mu
  const auto now = Clock::now();
  int off = 0;
  for (auto& r : sl.reqs) {
    if (status == BH_OK) {
      std::memcpy(r->r.quat_out, sl.h_quat + (size_t)off * 4, sizeof(float) * (size_t)r->r.B * 4);
      std::memcpy(r->r.score_out, sl.h_score + off, sizeof(float) * (size_t)r->r.B);
    }
    off += r->r.B;
    r->t_done = now;
    r->status = status;
    if (r->parent) {  // a piece: its outputs were written into the request's arrays
      Req& q = *r->parent;
      if (status != BH_OK) q.status = status;
      if (--q.pieces_left == 0) {
        q.t_done = now;
        if (q.status == BH_PENDING) q.status = BH_OK;
        ++s->completed;
      }
    } else {
      ++s->completed;
    }
  }
  sl.reqs.clear();
  sl.busy = false;
  s->used -= sl.bytes;
  sl.bytes = 0;
}

// The next piece of request q (caller holds s->mu): at most `piece` subtomograms from q.next_off on, with
// the request's arrays offset and, for random starts, the seed offset so that the piece draws the starts
// its subtomograms would draw unsplit (bh_random_starts counter seed + 3 (b S + s)).
std::shared_ptr<Req> next_piece(bh_server* s, const std::shared_ptr<Req>& q) {
  const int off = q->next_off, n = std::min(s->o.piece, q->r.B - off);
  const size_t N3 = (size_t)q->N * q->N * q->N;
  auto pc = std::make_shared<Req>();
  pc->ticket = 0;
  pc->r = q->r;
  pc->r.B = n;
  pc->r.vols = q->r.vols + (size_t)off * N3;
  pc->r.quat_out = q->r.quat_out + (size_t)off * 4;
  pc->r.score_out = q->r.score_out + off;
  if (q->r.starts)
    pc->r.starts = q->r.starts + (size_t)off * q->r.S * 4;
  else
    pc->r.seed = q->r.seed + 3ull * (uint64_t)off * (uint64_t)q->r.S;
  pc->N = q->N;
  pc->row = q->row;
  pc->express = q->express;
  pc->t_submit = q->t_submit;
  pc->parent = q;
  q->next_off = off + n;
  return pc;
}

void worker_loop(bh_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // 1. retire finished batches
    bool any_busy = false;
    for (auto& sl : s->slots) {
      if (!sl.busy) continue;
      cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      retire(s, sl, (e == cudaSuccess && sl.launch_status == BH_OK) ? BH_OK
                                                                    : (sl.launch_status != BH_OK ? sl.launch_status
                                                                                                 : BH_ERR_CUDA));
      s->cv_done.notify_all();
    }
    if (s->stop && !any_busy) break;
    // 2. admit: express first, then bulk; each class in its own arrival order
    bool launched = false;
    if (!s->stop && !s->paused && !s->queue.empty()) {
      bool bulk_waiting = false;
      for (auto& r : s->queue)
        if (!r->express) {
          bulk_waiting = true;
          break;
        }
      for (int cls = 1; cls >= 0 && !launched; --cls) {
        const bool ex = cls == 1;
        Slot* free_slot = nullptr;
        for (auto& sl : s->slots)
          if (!sl.busy && sl.express == ex) {
            free_slot = &sl;
            break;
          }
        if (!free_slot && ex && !bulk_waiting)
          for (auto& sl : s->slots)
            if (!sl.busy) {
              free_slot = &sl;
              break;
            }
        if (!free_slot) continue;
        std::shared_ptr<Req> head;
        for (auto& r : s->queue)
          if (r->express == ex) {
            head = r;
            break;
          }
        if (!head) continue;
        const int N = head->N, S = head->r.S;
        const Box& box = s->boxes[N];
        bh_plan* p = box.plan;
        std::vector<std::shared_ptr<Req>> take;
        std::vector<std::shared_ptr<Req>> next_pieces;
        int B = 0;
        for (auto it = s->queue.begin(); it != s->queue.end();) {
          auto& r = *it;
          if (r->express != ex) {
            ++it;
            continue;
          }
          const bool fits = r->N == N && r->r.S == S && B + r->r.B <= s->o.max_batch &&
                            s->used + batch_bytes(p, B + r->r.B, S, s->in_place) <= s->o.hbm_budget_bytes &&
                            (!ex || take.empty() ||
                             est_ms(p, box.stages, box.nstages, s->o.steps, B + r->r.B, S) <= s->express_ms);
          if (fits) {
            B += r->r.B;
            take.push_back(r);
            if (r->parent && r->parent->next_off < r->parent->r.B) next_pieces.push_back(next_piece(s, r->parent));
            it = s->queue.erase(it);
          } else if (take.empty()) {
            break;  // the class head does not fit yet: keep its arrival order
          } else {
            ++it;
          }
        }
        for (auto& pc : next_pieces) s->queue.push_back(pc);  // behind everything that arrived meanwhile
        if (take.empty()) continue;
        free_slot->busy = true;
        free_slot->reqs = take;
        free_slot->bytes = batch_bytes(p, B, S, s->in_place);
        s->used += free_slot->bytes;
        ++s->batches;
        if (ex) ++s->express_batches;
        if (s->in_place) ++s->in_place_batches;
        lk.unlock();
        int rc;
        const auto t_launch = Clock::now();
        {
          std::lock_guard<std::mutex> pg(s->plan_mu);
          rc = launch_batch(s, *free_slot, N, S);
        }
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t_launch).count();
        lk.lock();
        s->launch_ms_total += ms;
        s->launch_ms_max = std::max(s->launch_ms_max, ms);
        free_slot->launch_status = rc;
        if (rc != BH_OK) cudaEventRecord(free_slot->done, free_slot->stream);
        launched = true;
      }
    }
    if (!launched) s->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 2000));
  }
}

}  // namespace

using namespace bh;

extern "C" int bh_random_starts(uint64_t seed, int B, int S, float* out) {
  clear_error();
  if (B < 0 || S < 0 || (B > 0 && S > 0 && !out)) return fail(BH_ERR_ARG, "bad arguments");
  for (int b = 0; b < B; ++b)
    for (int s = 0; s < S; ++s) {
      const uint64_t c = seed + 3ull * ((uint64_t)b * S + s);
      double u[3];
      for (int j = 0; j < 3; ++j) u[j] = (double)(splitmix64(c + j) >> 11) * (1.0 / 9007199254740992.0);
      const double a = std::sqrt(1.0 - u[0]), bb = std::sqrt(u[0]);
      double q[4] = {bb * std::cos(2 * M_PI * u[2]), a * std::sin(2 * M_PI * u[1]), a * std::cos(2 * M_PI * u[1]),
                     bb * std::sin(2 * M_PI * u[2])};
      const double sg = q[0] < 0 ? -1.0 : 1.0;
      for (int j = 0; j < 4; ++j) out[((size_t)b * S + s) * 4 + j] = (float)(sg * q[j]);
    }
  return BH_OK;
}

extern "C" int bh_serve_create(bh_server** out, const bh_serve_opts* o) {
  clear_error();
  if (!out) return fail(BH_ERR_ARG, "out is NULL");
  *out = nullptr;
  bh_serve_opts opts{};
  if (o) opts = *o;
  if (opts.hbm_budget_bytes == 0) opts.hbm_budget_bytes = 8ull << 30;
  if (opts.max_inflight == 0) opts.max_inflight = 4;
  if (opts.max_batch == 0) opts.max_batch = 1024;
  if (opts.queue_capacity == 0) opts.queue_capacity = 65536;
  if (opts.steps == 0) opts.steps = 30;
  if (opts.ingest != 0 && opts.ingest != 1) return fail(BH_ERR_ARG, "ingest %d not in {0,1}", opts.ingest);
  if (opts.express_ms == 0.0) opts.express_ms = 2.0;
  if (opts.piece == 0) opts.piece = 128;
  if (opts.piece < 1) return fail(BH_ERR_ARG, "piece %d", opts.piece);
  if (opts.max_inflight < 1 || opts.max_inflight > 16) return fail(BH_ERR_ARG, "max_inflight %d", opts.max_inflight);
  if (opts.max_batch < 1 || opts.max_batch > 65536) return fail(BH_ERR_ARG, "max_batch %d", opts.max_batch);
  if (opts.queue_capacity < 1) return fail(BH_ERR_ARG, "queue_capacity %d", opts.queue_capacity);
  if (opts.steps < 0 || opts.steps > 100000) return fail(BH_ERR_ARG, "steps %d", opts.steps);
  if (opts.newton != 0 && opts.newton != 1) return fail(BH_ERR_ARG, "newton %d not in {0,1}", opts.newton);
  if (opts.mode != BH_MODE_FP32 && opts.mode != BH_MODE_BF16_SPLIT) return fail(BH_ERR_ARG, "mode %d", opts.mode);
  if (opts.express_slots < 0 || opts.express_slots > 16) return fail(BH_ERR_ARG, "express_slots %d", opts.express_slots);
  if (!(opts.express_ms > 0.0) || !std::isfinite(opts.express_ms)) return fail(BH_ERR_ARG, "express_ms %g", opts.express_ms);
  int dev = 0;
  BH_CUDA_TRY(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  BH_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  if (prop.major != 10 || prop.minor != 3) return fail(BH_ERR_UNSUPPORTED, "device is sm_%d%d", prop.major, prop.minor);
  int prio_low = 0, prio_high = 0;
  BH_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  auto* s = new bh_server();
  s->device = dev;
  s->o = opts;
  s->express_ms = opts.express_ms;
  int pageable = 0;
  BH_CUDA_TRY(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev));
  s->in_place = opts.ingest == 0 && pageable == 1;
  const int n_express = opts.express_slots;
  s->slots.resize(opts.max_inflight + n_express);
  for (size_t i = 0; i < s->slots.size(); ++i) {
    Slot& sl = s->slots[i];
    sl.express = (int)i >= opts.max_inflight;
    if (cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, sl.express ? prio_high : prio_low) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      bh_serve_destroy(s);
      return fail(BH_ERR_CUDA, "stream/event creation failed");
    }
  }
  for (auto& sl : s->slots)
    if (grow_staging(s, sl, opts.max_batch, kStagedStarts) != BH_OK) {
      bh_serve_destroy(s);
      return fail(BH_ERR_OOM, "pinned staging for %d subtomograms", opts.max_batch);
    }
  // the server's own stream-ordered pool: memory up to the budget stays mapped between batches
  cudaMemPoolProps pp{};
  pp.allocType = cudaMemAllocationTypePinned;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = dev;
  if (cudaMemPoolCreate(&s->pool, &pp) != cudaSuccess) {
    s->pool = nullptr;
    bh_serve_destroy(s);
    return fail(BH_ERR_CUDA, "memory pool creation failed");
  }
  // Memory freed by another stream's batch is reused only once that free has completed: the pool must
  // not make a batch wait on an unrelated one (an express batch would otherwise inherit the latency of
  // the bulk batch whose memory it was given).
  uint64_t keep = opts.hbm_budget_bytes;
  int no_dep = 0;
  if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
      cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no_dep) != cudaSuccess) {
    bh_serve_destroy(s);
    return fail(BH_ERR_CUDA, "memory pool attributes");
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return BH_OK;
}

extern "C" int bh_serve_add_template(bh_server* s, int N, const float* vol, int* template_id) {
  clear_error();
  if (!s || !vol || !template_id) return fail(BH_ERR_ARG, "NULL argument");
  if (N < 8 || N > 256 || N % 2) return fail(BH_ERR_ARG, "N=%d must be even in 8..256", N);
  BH_CUDA_TRY(cudaSetDevice(s->device));
  std::lock_guard<std::mutex> pg(s->plan_mu);
  Box* box;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    box = &s->boxes[N];
  }
  if (!box->plan) {
    bh_plan_opts po{};
    po.N = N;
    po.Lmax = N / 2;
    po.lambda_max = 0.0;
    po.mode = s->o.mode;
    po.max_batch = 128;
    int rc = bh_plan_create(&box->plan, &po);
    if (rc != BH_OK) return rc;
    box->N = N;
    BH_CUDA_TRY(cudaMalloc(&box->d_tmpl, sizeof(float) * 2 * (size_t)kMaxTemplatesPerBox * box->plan->Nb));
    const int L = N / 2;
    int cand[3] = {L / 4, L / 2, L};
    box->nstages = 0;
    for (int c : cand)
      if (c >= 1 && (box->nstages == 0 || c > box->stages[box->nstages - 1])) box->stages[box->nstages++] = c;
  }
  if (box->n_tmpl >= kMaxTemplatesPerBox) return fail(BH_ERR_ARG, "more than %d templates for N=%d", kMaxTemplatesPerBox, N);
  const size_t N3 = (size_t)N * N * N;
  float* d_vol = nullptr;
  BH_CUDA_TRY(cudaMalloc(&d_vol, N3 * sizeof(float)));
  cudaError_t e = cudaMemcpy(d_vol, vol, N3 * sizeof(float), cudaMemcpyHostToDevice);
  int rc = (e == cudaSuccess) ? BH_OK : fail(BH_ERR_CUDA, "template upload: %s", cudaGetErrorString(e));
  if (rc == BH_OK) rc = bh_expand(box->plan, d_vol, 1, box->d_tmpl + (size_t)2 * box->n_tmpl * box->plan->Nb, nullptr);
  if (rc == BH_OK && cudaDeviceSynchronize() != cudaSuccess) rc = fail(BH_ERR_CUDA, "template expansion failed");
  cudaFree(d_vol);
  if (rc != BH_OK) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  *template_id = (int)s->templates.size();
  s->templates.push_back({N, box->n_tmpl});
  box->n_tmpl++;
  return BH_OK;
}

extern "C" int bh_serve_submit(bh_server* s, const bh_request* r, uint64_t* ticket) {
  clear_error();
  if (!s || !r || !ticket) return fail(BH_ERR_ARG, "NULL argument");
  if (r->B < 1) return fail(BH_ERR_ARG, "B=%d", r->B);
  if (r->S < 1 || r->S > 512) return fail(BH_ERR_ARG, "S=%d outside 1..512", r->S);
  if (!r->vols || !r->quat_out || !r->score_out) return fail(BH_ERR_ARG, "NULL request array");
  std::lock_guard<std::mutex> lk(s->mu);
  if (r->template_id < 0 || r->template_id >= (int)s->templates.size())
    return fail(BH_ERR_ARG, "unknown template %d", r->template_id);
  const Template t = s->templates[r->template_id];
  const bh_plan* p = s->boxes[t.N].plan;
  if (r->B > s->o.max_batch) return fail(BH_ERR_BUDGET, "B=%d exceeds max_batch %d", r->B, s->o.max_batch);
  if (batch_bytes(p, r->B, r->S, s->in_place) > s->o.hbm_budget_bytes)
    return fail(BH_ERR_BUDGET, "request needs %zu device bytes, budget %zu", batch_bytes(p, r->B, r->S, s->in_place),
                s->o.hbm_budget_bytes);
  if ((int)s->queue.size() >= s->o.queue_capacity) return fail(BH_ERR_BUSY, "queue full");
  auto q = std::make_shared<Req>();
  q->ticket = s->next_ticket++;
  q->r = *r;
  q->N = t.N;
  q->row = t.row;
  const Box& box = s->boxes[t.N];
  q->express = s->o.express_slots > 0 &&
               est_ms(p, box.stages, box.nstages, s->o.steps, std::min(r->B, s->o.piece), r->S) <= s->express_ms;
  q->t_submit = Clock::now();
  if (r->B > s->o.piece) {  // admitted piece by piece; the first piece is queued now
    q->pieces_left = (r->B + s->o.piece - 1) / s->o.piece;
    s->queue.push_back(next_piece(s, q));
  } else {
    s->queue.push_back(q);
  }
  s->reqs[q->ticket] = q;
  ++s->submitted;
  *ticket = q->ticket;
  s->cv_work.notify_one();
  return BH_OK;
}

static int poll_locked(bh_server* s, uint64_t ticket, double* latency_ms) {
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(BH_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  auto& r = it->second;
  if (r->status == BH_PENDING) return BH_PENDING;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  return r->status == BH_OK ? BH_OK : fail(r->status, "batch failed (status %d)", r->status);
}

extern "C" int bh_serve_poll(bh_server* s, uint64_t ticket, double* latency_ms) {
  clear_error();
  if (!s) return fail(BH_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  return poll_locked(s, ticket, latency_ms);
}

extern "C" int bh_serve_wait(bh_server* s, uint64_t ticket, double timeout_ms, double* latency_ms) {
  clear_error();
  if (!s) return fail(BH_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1000.0));
  for (;;) {
    int st = poll_locked(s, ticket, latency_ms);
    if (st != BH_PENDING) return st;
    if (timeout_ms >= 0 && Clock::now() >= deadline)
      return fail(BH_ERR_TIMEOUT, "ticket %llu not finished after %.1f ms", (unsigned long long)ticket, timeout_ms);
    if (timeout_ms >= 0)
      s->cv_done.wait_until(lk, deadline);
    else
      s->cv_done.wait_for(lk, std::chrono::milliseconds(100));
  }
}

extern "C" int bh_serve_pause(bh_server* s, int paused) {
  clear_error();
  if (!s) return fail(BH_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  s->paused = paused != 0;
  s->cv_work.notify_one();
  return BH_OK;
}

extern "C" int bh_serve_stats(bh_server* s, bh_serve_counters* out) {
  clear_error();
  if (!s || !out) return fail(BH_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->express_batches = s->express_batches;
  out->in_place_batches = s->in_place_batches;
  out->staging_allocs = s->staging_allocs.load();
  out->launch_ms_total = s->launch_ms_total;
  out->launch_ms_max = s->launch_ms_max;
  out->queued = s->queue.size();
  out->inflight_batches = 0;
  for (auto& sl : s->slots) out->inflight_batches += sl.busy ? 1 : 0;
  out->inflight_bytes = s->used;
  return BH_OK;
}

extern "C" int bh_serve_destroy(bh_server* s) {
  clear_error();
  if (!s) return BH_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& q : s->queue) {
      q->status = BH_ERR_ARG;
      if (q->parent) q->parent->status = BH_ERR_ARG;
    }
    s->queue.clear();
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (auto& sl : s->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
    cudaFreeHost(sl.h_starts);
    cudaFreeHost(sl.h_tidx);
    cudaFreeHost(sl.h_quat);
    cudaFreeHost(sl.h_score);
    cudaFreeHost(sl.h_vptr);
  }
  for (auto& kv : s->boxes) {
    cudaFree(kv.second.d_tmpl);
    bh_plan_destroy(kv.second.plan);
  }
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
  return BH_OK;
}
