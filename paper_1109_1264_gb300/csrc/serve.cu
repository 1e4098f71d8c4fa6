// Serving loop (include/salt.h, salt_serve_*): continuous batching of
// expression requests on one GPU.
//
// Requests arrive at any time.  A scheduler thread admits them in arrival
// order while resident slots and the device-memory budget allow (operand
// vectors live in a device arena until the client releases the request), and
// launches a step as soon as one of its streams is free: every request
// admitted since the previous step goes into ONE batched launch pair -- a fill
// launch that writes the requests' input vectors on the device (standing in
// for their upload), then the compute launch.  Requests arriving while steps
// run wait for the next free stream, so up to `streams` steps overlap on the
// GPU.  Completion is observed by polling each step's event; a request's
// latency is completion time minus submission time on the host clock.
//
// Every request runs with the same tile size, so its reductions use the same
// partition whatever else is in its step: alone or in a mix, the results are
// the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/salt.h"
#include "batch.cuh"
#include "internal.h"
#include "persist.cuh"
#include "registry.h"

using namespace salt;

namespace {

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
// After its last step the scheduler keeps polling (yielding) this long before
// it sleeps on the condition variable: waking a sleeping thread costs several
// microseconds, which the next arrival would pay in its latency.
constexpr double kIdleSpinUs = 1000.0;
size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, size) with coalescing of freed neighbours.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
    size_ = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t start = it->first, rem = it->second - bytes;
        free_.erase(it);
        if (rem) free_[start + bytes] = rem;
        used_ += bytes;
        *off = start;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

enum : int32_t { RS_WAITING = 0, RS_RUNNING = 1, RS_DONE = 2 };

struct Request {
  int64_t id = 0;
  int32_t kind = 0;  // shape id or kKindNrm2
  int32_t dtype = 0;
  int64_t n = 0;
  int nvec = 0;
  uint32_t load_mask = 0;
  int nred = 0;
  uint64_t keys[kBatchOps] = {0, 0, 0, 0, 0};
  int user_of[kBatchOps] = {0, 0, 0, 0, 0};  // canonical operand -> user operand index
  double sc[2] = {0.0, 0.0};
  size_t vec_bytes = 0;
  size_t off[kBatchOps] = {0, 0, 0, 0, 0};
  char* ext[kBatchOps] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // caller-owned operand, or NULL
  bool resident = false;
  int32_t state = RS_WAITING;
  double t_submit = 0, t_done = 0;
  double red[kBatchPartials] = {0, 0, 0};
  int64_t bytes_alg = 0;  // algorithmic bytes of the compute
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* d_mem = nullptr;
  char* h_mem = nullptr;
  // device layout: the tables (packed per step at the start of d_mem), then
  // the per-table tile counters, the partials and the results
  unsigned* d_counters[2] = {nullptr, nullptr};
  double* d_partials = nullptr;
  // host staging (pinned): the packed tables, then red
  size_t table_bytes = 0;
  std::vector<BatchItem> compute_items;  // built aside, copied after the fill items
  double* h_red = nullptr;      // pinned and mapped: the kernel writes the results here
  double* h_red_dev = nullptr;  // its device address
  std::vector<Request*> reqs;
  bool busy = false;
  // The step as one CUDA graph: table upload -> [fill launch ->] compute
  // launch, instantiated once with and once without the fill launch; each
  // step updates the upload size and launch parameters of one of them and
  // replays it.  No reset or read-back nodes: the batch kernel leaves its
  // counters at zero, and writes the results straight into mapped pinned
  // host memory.
  struct StepGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t n_up = nullptr, n_fill = nullptr, n_comp = nullptr;
  } g[2];  // [0] without, [1] with the fill launch
};

using KernelFn = void (*)(const BatchParams);
KernelFn kernel_for(int unroll) {
  switch (unroll) {
    case 1: return &batch_kernel<1>;
    case 2: return &batch_kernel<2>;
    default: return &batch_kernel<4>;
  }
}

using PersistFn = void (*)(const PersistParams);
PersistFn persist_for(int unroll) {
  switch (unroll) {
    case 1: return &persist_kernel<1>;
    case 2: return &persist_kernel<2>;
    default: return &persist_kernel<4>;
  }
}

// Bound on the waits of the persistent kernel other than block 0's wait for
// a posted step (which the configuration's idle time bounds).
constexpr unsigned long long kPersistWaitNs = 1000000000ull;
std::atomic<unsigned> g_serve_polls{67108864u};

// Persistent mode (salt_serve_config.persistent): steps are posted to a ring
// of `streams` entries in mapped pinned host memory and run by one resident
// launch of persist_kernel (persist.cuh) until it has been idle for idle_us.
struct PersistState {
  bool on = false;
  int nring = 0;
  int grid = 0;
  PersistCtl* ctl = nullptr;  // mapped pinned host memory
  PersistCtl* ctl_dev = nullptr;
  char* ring = nullptr;       // nring entries of entry_bytes, mapped
  char* ring_dev = nullptr;
  size_t entry_bytes = 0;
  double* red = nullptr;      // nring x red_stride results, mapped
  double* red_dev = nullptr;
  size_t red_stride = 0;
  char* d_mem = nullptr;      // device: 2 tables (entry_bytes each) | 4 counter sets | 2 partials | sync words
  size_t off_counters = 0, off_partials = 0, off_sync = 0, counters_stride = 0, partials_stride = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ended = nullptr;  // recorded after each launch
  std::atomic<bool> live{false};
  std::atomic<int64_t> launches{0};
  uint64_t epoch = 0, posted = 0;
  struct Entry {
    std::vector<Request*> reqs;
    uint64_t step = 0;
  };
  std::deque<Entry> inflight;  // posted and not complete, in step order
  std::vector<BatchItem> comps;
};

salt_status fail(salt_status st, const std::string& m) { return report_error(st, m); }
salt_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SALT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

struct salt_server {
  salt_serve_config cfg{};
  int device = 0;
  int sms = 0;
  int grid = 0;
  char* arena_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  PersistState ps;
  int64_t items_cap = 0, tiles_cap = 0;
  // shared state
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> waiting;             // submitted, not yet admitted
  std::deque<Request*> pending;             // admitted (resident), not yet launched
  std::unordered_map<int64_t, Request*> reqs;
  std::deque<int64_t> completed;            // completion queue (ids)
  int64_t next_id = 1;
  int32_t resident = 0;
  bool stop = false;
  std::thread sched;
  std::string sched_error;
  // statistics
  std::atomic<int64_t> n_done{0}, n_steps{0}, bytes_done{0};
};

namespace {

size_t slot_device_bytes(const salt_server* s, size_t* off_items, size_t* off_counters, size_t* off_partials) {
  const size_t hdr = 256;
  const size_t items = round_up(sizeof(BatchItem) * (size_t)s->items_cap);
  // tile counter, finished blocks, per-item tickets
  const size_t counters = round_up(sizeof(unsigned) * (size_t)(s->items_cap + 2));
  const size_t partials = round_up(sizeof(double) * kBatchPartials * (size_t)s->tiles_cap);
  // [hdr0 items0 hdr1 items1 | counters0 counters1 | partials]
  off_items[0] = hdr;
  off_items[1] = hdr + items + hdr;
  off_counters[0] = 2 * (hdr + items);
  off_counters[1] = off_counters[0] + counters;
  *off_partials = off_counters[1] + counters;
  return *off_partials + partials;
}

// Called with the request's shape/dtype set: lay out its operands in the arena.
// Caller-owned operands take no arena space.
bool arena_take(salt_server* s, Request* r) {
  int k = 0;
  for (; k < r->nvec; ++k) {
    if (r->ext[k]) continue;
    if (!s->arena.alloc(r->vec_bytes, &r->off[k])) break;
  }
  if (k == r->nvec) return true;
  for (int j = 0; j < k; ++j)
    if (!r->ext[j]) s->arena.release(r->off[j], r->vec_bytes);
  return false;
}

void arena_give(salt_server* s, Request* r) {
  for (int k = 0; k < r->nvec; ++k)
    if (!r->ext[k]) s->arena.release(r->off[k], r->vec_bytes);
}

char* operand_ptr(const salt_server* s, const Request* r, int k) {
  return r->ext[k] ? r->ext[k] : s->arena_base + r->off[k];
}

int64_t tiles_of(const salt_server* s, int dtype, int64_t n) {
  const int64_t te = s->cfg.tile_bytes / (dtype == SALT_F32 ? 4 : 8);
  return n > 0 ? (n + te - 1) / te : 1;
}

// Builds a step graph with placeholder sizes and launch shapes (every step
// sets its own before replaying it).
cudaError_t build_step_graph(salt_server* s, Slot& slot, bool with_fill, Slot::StepGraph* sg) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  e = cudaGraphAddMemcpyNode1D(&sg->n_up, g, nullptr, 0, slot.d_mem, slot.h_mem, 512, cudaMemcpyHostToDevice);
  BatchParams prm{(BatchHeader*)slot.d_mem, (BatchItem*)(slot.d_mem + 512), slot.d_counters[0],
                  slot.d_counters[0] + 1, slot.d_counters[0] + 2, slot.d_partials, slot.h_red_dev};
  void* args[] = {&prm};
  cudaKernelNodeParams kp{};
  kp.func = (void*)kernel_for(s->cfg.unroll);
  kp.gridDim = dim3(1);
  kp.blockDim = dim3((unsigned)s->cfg.block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaGraphNode_t before = sg->n_up;
  if (e == cudaSuccess && with_fill) {
    e = cudaGraphAddKernelNode(&sg->n_fill, g, &before, 1, &kp);
    before = sg->n_fill;
  }
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&sg->n_comp, g, &before, 1, &kp);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&sg->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  sg->graph = g;
  return cudaSuccess;
}

// The item tables of one step: a fill item per server-owned input operand
// (fills[0 .. nitems[0])) and a compute item per request (comps[0 ..
// nitems[1])), with their global tile numbers and result slots.
void build_items(const salt_server* s, const std::vector<Request*>& batch, BatchItem* fills, BatchItem* comps,
                 int (&nitems)[2], int64_t (&tiles)[2]) {
  nitems[0] = nitems[1] = 0;
  tiles[0] = tiles[1] = 0;
  int nred = 0;
  for (Request* r : batch) {
    const int dt = r->dtype == SALT_F32 ? DT_F32 : DT_F64;
    for (int k = 0; k < r->nvec; ++k) {
      if (!((r->load_mask >> k) & 1u) || r->ext[k]) continue;  // caller-owned inputs are already there
      BatchItem& f = fills[nitems[0]++];
      memset(&f, 0, sizeof f);
      f.kind = kKindFill;
      f.dtype = dt;
      f.n = r->n;
      f.tile_begin = tiles[0];
      f.ntiles = (int32_t)tiles_of(s, r->dtype, r->n);
      f.red_index = -1;
      f.v[0] = operand_ptr(s, r, k);
      uint64_t key = r->keys[k];
      memcpy(&f.sc[0], &key, sizeof key);
      tiles[0] += f.ntiles;
    }
    BatchItem& c = comps[nitems[1]++];
    memset(&c, 0, sizeof c);
    c.kind = r->kind;
    c.dtype = dt;
    c.n = r->n;
    c.tile_begin = tiles[1];
    c.ntiles = (int32_t)tiles_of(s, r->dtype, r->n);
    c.red_index = r->nred > 0 ? nred : -1;
    for (int k = 0; k < r->nvec; ++k) c.v[k] = operand_ptr(s, r, k);
    c.sc[0] = r->sc[0];
    c.sc[1] = r->sc[1];
    tiles[1] += c.ntiles;
    nred += r->nred;
  }
}

// Builds and launches one step on `slot` from the front of `pending`
// (scheduler thread, lock not held while launching).
salt_status launch_step(salt_server* s, Slot& slot, std::vector<Request*>& batch) {
  size_t off_items[2], off_counters[2], off_partials;
  slot_device_bytes(s, off_items, off_counters, &off_partials);
  // Host tables in the pinned staging area, packed so that one copy of
  // only the bytes in use moves them: [hdr0 | hdr1 | fill items | compute
  // items].  Compute items are built aside, then placed after the fills.
  BatchHeader* h_hdr[2] = {(BatchHeader*)slot.h_mem, (BatchHeader*)(slot.h_mem + 256)};
  BatchItem* h_items[2] = {(BatchItem*)(slot.h_mem + 512), slot.compute_items.data()};
  int nitems[2];
  int64_t tiles[2];
  build_items(s, batch, h_items[0], h_items[1], nitems, tiles);
  const size_t off_compute = 512 + round_up(sizeof(BatchItem) * (size_t)nitems[0]);
  memcpy(slot.h_mem + off_compute, slot.compute_items.data(), sizeof(BatchItem) * (size_t)nitems[1]);
  const size_t used = off_compute + sizeof(BatchItem) * (size_t)nitems[1];
  for (int t = 0; t < 2; ++t) {
    memset(h_hdr[t], 0, sizeof(BatchHeader));
    h_hdr[t]->nitems = nitems[t];
    h_hdr[t]->total_tiles = tiles[t];
    h_hdr[t]->tile_bytes = s->cfg.tile_bytes;
  }
  BatchHeader* d_hdr[2] = {(BatchHeader*)slot.d_mem, (BatchHeader*)(slot.d_mem + 256)};
  BatchItem* d_items[2] = {(BatchItem*)(slot.d_mem + 512), (BatchItem*)(slot.d_mem + off_compute)};
  KernelFn k = kernel_for(s->cfg.unroll);
  BatchParams prm[2];
  cudaKernelNodeParams kp[2];
  for (int t = 0; t < 2; ++t) {
    prm[t] = BatchParams{d_hdr[t], d_items[t], slot.d_counters[t], slot.d_counters[t] + 1,
                         slot.d_counters[t] + 2, slot.d_partials, slot.h_red_dev};
    kp[t] = cudaKernelNodeParams{};
    kp[t].func = (void*)k;
    kp[t].gridDim = dim3((unsigned)std::max<int64_t>(1, std::min<int64_t>(s->grid, tiles[t])));
    kp[t].blockDim = dim3((unsigned)s->cfg.block);
    kp[t].sharedMemBytes = 0;
    kp[t].extra = nullptr;
  }
  void* args0[] = {&prm[0]};
  void* args1[] = {&prm[1]};
  kp[0].kernelParams = args0;
  kp[1].kernelParams = args1;
  Slot::StepGraph& sg = slot.g[nitems[0] > 0 ? 1 : 0];
  cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(sg.exec, sg.n_up, slot.d_mem, slot.h_mem, used,
                                                     cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nitems[0] > 0) e = cudaGraphExecKernelNodeSetParams(sg.exec, sg.n_fill, &kp[0]);
  if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(sg.exec, sg.n_comp, &kp[1]);
  if (e == cudaSuccess) e = cudaGraphLaunch(sg.exec, slot.stream);
  if (e == cudaSuccess) {
    if (nitems[0] > 0) count_launch();
    count_launch();
  }
  if (e == cudaSuccess) e = cudaEventRecord(slot.done, slot.stream);
  if (e != cudaSuccess) return cuda_fail(e, "serving step");
  slot.reqs = batch;
  slot.busy = true;
  s->n_steps.fetch_add(1);
  return SALT_OK;
}

void complete_slot(salt_server* s, Slot& slot) {
  const double t = now_us();
  std::lock_guard<std::mutex> lk(s->mu);
  int idx = 0;
  for (Request* r : slot.reqs) {
    for (int j = 0; j < r->nred; ++j) r->red[j] = slot.h_red[idx + j];
    idx += r->nred;
    r->state = RS_DONE;
    r->t_done = t;
    s->completed.push_back(r->id);
    s->n_done.fetch_add(1);
    s->bytes_done.fetch_add(r->bytes_alg);
  }
  slot.reqs.clear();
  slot.busy = false;
  s->cv.notify_all();
}

// ---------------------------------------------------------- persistent ---

void persist_free(salt_server* s) {
  PersistState& ps = s->ps;
  if (ps.stream) cudaStreamSynchronize(ps.stream);
  if (ps.d_mem) cudaFree(ps.d_mem);
  if (ps.ring) cudaFreeHost(ps.ring);
  if (ps.red) cudaFreeHost(ps.red);
  if (ps.ctl) cudaFreeHost(ps.ctl);
  if (ps.ended) cudaEventDestroy(ps.ended);
  if (ps.stream) cudaStreamDestroy(ps.stream);
  ps.d_mem = ps.ring = nullptr;
  ps.red = nullptr;
  ps.ctl = nullptr;
  ps.ended = nullptr;
  ps.stream = nullptr;
}

salt_status persist_init(salt_server* s) {
  PersistState& ps = s->ps;
  int coop = 0;
  cudaError_t e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, s->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (!coop) return fail(SALT_ERR_CUDA, "persistent serving needs cooperative launches");
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)persist_for(s->cfg.unroll), s->cfg.block, 0);
  if (e != cudaSuccess) return cuda_fail(e, "persistent kernel occupancy");
  if (bps < 1) return fail(SALT_ERR_CUDA, "the persistent kernel does not fit on an SM");
  ps.grid = s->sms * bps;
  ps.nring = s->cfg.streams;
  ps.entry_bytes = round_up((size_t)(kStepHead + 2 * kHdrSlot) +
                            sizeof(BatchItem) * (size_t)(s->items_cap + s->cfg.max_batch) + 32);
  ps.red_stride = (size_t)kBatchPartials * (size_t)s->cfg.max_batch;
  ps.counters_stride = (size_t)s->items_cap + 2;
  ps.partials_stride = (size_t)kBatchPartials * (size_t)s->tiles_cap;
  ps.off_counters = 2 * ps.entry_bytes;
  ps.off_partials = ps.off_counters + round_up(sizeof(unsigned) * 4 * ps.counters_stride);
  ps.off_sync = ps.off_partials + round_up(sizeof(double) * 2 * ps.partials_stride);
  const size_t dbytes = ps.off_sync + kAlign;
  e = cudaHostAlloc(&ps.ctl, sizeof(PersistCtl), cudaHostAllocMapped);
  if (e == cudaSuccess) {
    memset(ps.ctl, 0, sizeof(PersistCtl));
    e = cudaHostGetDevicePointer((void**)&ps.ctl_dev, ps.ctl, 0);
  }
  if (e == cudaSuccess) e = cudaHostAlloc(&ps.ring, ps.entry_bytes * (size_t)ps.nring, cudaHostAllocMapped);
  if (e == cudaSuccess) {
    memset(ps.ring, 0, ps.entry_bytes * (size_t)ps.nring);
    e = cudaHostGetDevicePointer((void**)&ps.ring_dev, ps.ring, 0);
  }
  if (e == cudaSuccess) e = cudaHostAlloc(&ps.red, sizeof(double) * ps.red_stride * (size_t)ps.nring, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&ps.red_dev, ps.red, 0);
  if (e == cudaSuccess) e = cudaMalloc(&ps.d_mem, dbytes);
  // counters and sync words start at zero; every step leaves the counters at zero
  if (e == cudaSuccess) e = cudaMemset(ps.d_mem, 0, dbytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ps.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ps.ended, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    persist_free(s);
    return cuda_fail(e, "persistent serving resources");
  }
  ps.comps.resize((size_t)s->cfg.max_batch);
  ps.on = true;
  return SALT_OK;
}

// Writes the step's tables into its ring entry and posts it (scheduler
// thread; the entry is free: fewer than nring steps are in flight).
void post_step(salt_server* s, std::vector<Request*>& batch) {
  PersistState& ps = s->ps;
  const uint64_t step = ps.posted + 1;
  char* base = ps.ring + (size_t)((step - 1) % (uint64_t)ps.nring) * ps.entry_bytes;
  StepDesc* d = (StepDesc*)base;
  BatchHeader* hdr[2] = {(BatchHeader*)(base + kStepHead), (BatchHeader*)(base + kStepHead + kHdrSlot)};
  const size_t off0 = (size_t)(kStepHead + 2 * kHdrSlot);
  int nitems[2];
  int64_t tiles[2];
  build_items(s, batch, (BatchItem*)(base + off0), ps.comps.data(), nitems, tiles);
  const size_t off1 = off0 + (sizeof(BatchItem) * (size_t)nitems[0] + 15) / 16 * 16;
  memcpy(base + off1, ps.comps.data(), sizeof(BatchItem) * (size_t)nitems[1]);
  for (int t = 0; t < 2; ++t) {
    memset(hdr[t], 0, sizeof(BatchHeader));
    hdr[t]->nitems = nitems[t];
    hdr[t]->total_tiles = tiles[t];
    hdr[t]->tile_bytes = s->cfg.tile_bytes;
  }
  d->off_items[0] = off0;
  d->off_items[1] = off1;
  d->used = (off1 + sizeof(BatchItem) * (size_t)nitems[1] + 15) / 16 * 16;
  // the entry's bytes before the step number that publishes them
  __atomic_thread_fence(__ATOMIC_SEQ_CST);
  __atomic_store_n(&ps.ctl->posted, (unsigned long long)step, __ATOMIC_RELEASE);
  ps.posted = step;
  ps.inflight.push_back(PersistState::Entry{batch, step});
  s->n_steps.fetch_add(1);
}

// Starts a launch of the persistent kernel at the first step not complete.
salt_status launch_persist(salt_server* s) {
  PersistState& ps = s->ps;
  PersistParams prm{};
  prm.ctl = ps.ctl_dev;
  prm.ring = ps.ring_dev;
  prm.entry_bytes = ps.entry_bytes;
  prm.red = ps.red_dev;
  prm.red_stride = ps.red_stride;
  prm.nring = (unsigned long long)ps.nring;
  prm.table = ps.d_mem;
  prm.counters = (unsigned*)(ps.d_mem + ps.off_counters);
  prm.counters_stride = ps.counters_stride;
  prm.partials = (double*)(ps.d_mem + ps.off_partials);
  prm.partials_stride = ps.partials_stride;
  prm.sync = (unsigned long long*)(ps.d_mem + ps.off_sync);
  prm.first_step = __atomic_load_n(&ps.ctl->done, __ATOMIC_ACQUIRE) + 1;
  prm.epoch = ++ps.epoch;
  prm.idle_ns = (unsigned long long)s->cfg.idle_us * 1000ull;
  prm.wait_ns = kPersistWaitNs;
  prm.max_polls = g_serve_polls.load();
  void* args[] = {&prm};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)persist_for(s->cfg.unroll), dim3((unsigned)ps.grid),
                                              dim3((unsigned)s->cfg.block), args, 0, ps.stream);
  if (e == cudaSuccess) e = cudaEventRecord(ps.ended, ps.stream);
  if (e != cudaSuccess) return cuda_fail(e, "persistent serving kernel");
  count_launch();
  ps.live.store(true);
  ps.launches.fetch_add(1);
  return SALT_OK;
}

void complete_entry(salt_server* s, const PersistState::Entry& en) {
  const double t = now_us();
  const double* red = s->ps.red + (size_t)((en.step - 1) % (uint64_t)s->ps.nring) * s->ps.red_stride;
  std::lock_guard<std::mutex> lk(s->mu);
  int idx = 0;
  for (Request* r : en.reqs) {
    for (int j = 0; j < r->nred; ++j) r->red[j] = red[idx + j];
    idx += r->nred;
    r->state = RS_DONE;
    r->t_done = t;
    s->completed.push_back(r->id);
    s->n_done.fetch_add(1);
    s->bytes_done.fetch_add(r->bytes_alg);
  }
  s->cv.notify_all();
}

// The scheduler of persistent mode: the same admission and batching as
// `scheduler`, with ring entries in place of streams.  Completions are read
// from the control block (in step order); a launch that has ended (idle, or
// the host's stop) is replaced when a posted step is not complete.
void scheduler_persist(salt_server* s) {
  cudaSetDevice(s->device);
  PersistState& ps = s->ps;
  std::vector<Request*> batch;
  double last_active = now_us();
  for (;;) {
    bool did = false;
    std::string err;
    if (ps.live.load()) {
      const cudaError_t q = cudaEventQuery(ps.ended);
      if (q == cudaSuccess) ps.live.store(false);
      else if (q != cudaErrorNotReady) err = std::string("persistent serving kernel failed: ") + cudaGetErrorString(q);
    }
    const uint64_t done = __atomic_load_n(&ps.ctl->done, __ATOMIC_ACQUIRE);
    while (!ps.inflight.empty() && ps.inflight.front().step <= done) {
      complete_entry(s, ps.inflight.front());
      ps.inflight.pop_front();
      did = true;
    }
    if (err.empty() && __atomic_load_n(&ps.ctl->status, __ATOMIC_ACQUIRE) != 0u)
      err = "persistent serving kernel: a bounded wait ran out in step " +
            std::to_string(__atomic_load_n(&ps.ctl->fail_step, __ATOMIC_ACQUIRE));
    if (err.empty() && !ps.live.load() && ps.posted > done) {
      const salt_status st = launch_persist(s);
      if (st != SALT_OK) err = salt_last_error();
    }
    if (!err.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->sched_error = err;
      s->stop = true;
      s->cv.notify_all();
      break;
    }
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (!s->waiting.empty() && s->resident < s->cfg.max_requests) {
        Request* r = s->waiting.front();
        if (!arena_take(s, r)) break;
        s->waiting.pop_front();
        r->resident = true;
        ++s->resident;
        s->pending.push_back(r);
      }
      const bool any_busy = !ps.inflight.empty();
      if (s->stop && !any_busy) break;
      if ((int)ps.inflight.size() < ps.nring && !s->pending.empty() && !s->stop) {
        int64_t tiles = 0, fills = 0;
        while (!s->pending.empty() && (int32_t)batch.size() < s->cfg.max_batch) {
          Request* r = s->pending.front();
          const int64_t t = tiles_of(s, r->dtype, r->n);
          int nf = 0;
          for (int k = 0; k < r->nvec; ++k) nf += ((r->load_mask >> k) & 1u) && !r->ext[k];
          if (!batch.empty() && (tiles + t > s->tiles_cap || fills + nf > s->items_cap)) break;
          s->pending.pop_front();
          r->state = RS_RUNNING;
          batch.push_back(r);
          tiles += t;
          fills += nf;
        }
      }
      if (batch.empty() && !did) {
        if (any_busy || now_us() - last_active < kIdleSpinUs) {
          lk.unlock();
          std::this_thread::yield();
        } else {
          s->cv.wait_for(lk, std::chrono::microseconds(200));
        }
        continue;
      }
    }
    last_active = now_us();
    if (!batch.empty()) {
      post_step(s, batch);
      if (!ps.live.load()) {
        const salt_status st = launch_persist(s);
        if (st != SALT_OK) {
          std::lock_guard<std::mutex> lk(s->mu);
          s->sched_error = salt_last_error();
          s->stop = true;
          s->cv.notify_all();
          break;
        }
      }
    }
  }
  // a live launch ends at its next look at the ring
  __atomic_store_n(&ps.ctl->stop, 1u, __ATOMIC_RELEASE);
}

void scheduler(salt_server* s) {
  cudaSetDevice(s->device);
  std::vector<Request*> batch;
  double last_active = now_us();
  for (;;) {
    bool did = false;
    for (Slot& slot : s->slots) {
      if (slot.busy) {
        const cudaError_t q = cudaEventQuery(slot.done);
        if (q == cudaSuccess) {
          complete_slot(s, slot);
          did = true;
        } else if (q != cudaErrorNotReady) {
          std::lock_guard<std::mutex> lk(s->mu);
          s->sched_error = std::string("step failed: ") + cudaGetErrorString(q);
          s->stop = true;
          s->cv.notify_all();
        }
      }
    }
    Slot* free_slot = nullptr;
    for (Slot& slot : s->slots)
      if (!slot.busy) {
        free_slot = &slot;
        break;
      }
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // admission: arrival order, while slots and budget allow
      while (!s->waiting.empty() && s->resident < s->cfg.max_requests) {
        Request* r = s->waiting.front();
        if (!arena_take(s, r)) break;
        s->waiting.pop_front();
        r->resident = true;
        ++s->resident;
        s->pending.push_back(r);
      }
      bool any_busy = false;
      for (Slot& slot : s->slots) any_busy = any_busy || slot.busy;
      if (s->stop && !any_busy) break;
      if (free_slot && !s->pending.empty() && !s->stop) {
        int64_t tiles = 0, fills = 0;
        while (!s->pending.empty() && (int32_t)batch.size() < s->cfg.max_batch) {
          Request* r = s->pending.front();
          const int64_t t = tiles_of(s, r->dtype, r->n);
          int nf = 0;
          for (int k = 0; k < r->nvec; ++k) nf += ((r->load_mask >> k) & 1u) && !r->ext[k];
          if (!batch.empty() && (tiles + t > s->tiles_cap || fills + nf > s->items_cap)) break;
          s->pending.pop_front();
          r->state = RS_RUNNING;
          batch.push_back(r);
          tiles += t;
          fills += nf;
        }
      }
      if (batch.empty() && !did) {
        if (any_busy || now_us() - last_active < kIdleSpinUs) {
          // A step is in flight, or one ended moments ago: poll again at once
          // (a timed wait of a few microseconds sleeps for the kernel's timer
          // slack, tens of microseconds, which would show up in every latency).
          lk.unlock();
          std::this_thread::yield();
        } else {
          s->cv.wait_for(lk, std::chrono::microseconds(200));  // idle: woken by submit
        }
        continue;
      }
    }
    last_active = now_us();
    if (!batch.empty()) {
      salt_status st = launch_step(s, *free_slot, batch);
      if (st != SALT_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->sched_error = salt_last_error();
        s->stop = true;
        s->cv.notify_all();
      }
    }
  }
}

// Key of operand `slot` of request `item` under `seed` (same recipe as the
// Python input module's vector_key).
uint64_t vector_key(uint64_t seed, uint64_t item, uint64_t slot) {
  return seed * 0x100000001B3ull + item * 16ull + slot + 1ull;
}

// Store vector and element offset of input operand k of replayed request i
// (salt_serve_replay_store): vector (5 i + k) mod count, offset a multiple of
// 32 bytes (`align` elements) in [0, len - n], spread by a multiplicative
// hash of the operand's key.
int32_t store_vector(int64_t i, int k, int32_t count) { return (int32_t)(((uint64_t)i * 5u + (uint64_t)k) % (uint64_t)count); }
int64_t store_offset(uint64_t seed, uint64_t i, uint64_t k, int64_t n, int64_t len, int64_t align) {
  const uint64_t h = (vector_key(seed, i, k) * 0x9E3779B97F4A7C15ull) >> 11;
  const int64_t o = (int64_t)(h % (uint64_t)(len - n + 1));
  return o - o % align;
}

salt_status submit_impl(salt_server* s, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                        const void* const* ptrs, const uint64_t* keys, int32_t nkeys, const double* scalars,
                        int32_t nscal, double t_submit, int64_t* id_out) {
  if (dtype != SALT_F32 && dtype != SALT_F64) return fail(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  if (n < 0 || n > s->cfg.max_n) return fail(SALT_ERR_ARG, "n outside 0 .. max_n of the server");
  if (nkeys < 0 || nkeys > kBatchOps || (nkeys > 0 && !keys && !ptrs)) return fail(SALT_ERR_ARG, "bad keys");
  for (int k = 0; ptrs && k < nkeys; ++k)
    if (ptrs[k] && (uintptr_t)ptrs[k] % 16) return fail(SALT_ERR_ALIGN, "caller-owned operands must be 16-byte aligned");
  Request* r = new Request();
  r->dtype = dtype;
  r->n = n;
  const int64_t es = dtype == SALT_F32 ? 4 : 8;
  if (!prog) {  // Euclidean norm of one operand
    if (nkeys != 1) {
      delete r;
      return fail(SALT_ERR_ARG, "a norm request has exactly one key");
    }
    r->kind = kKindNrm2;
    r->nvec = 1;
    r->load_mask = 1u;
    r->nred = 1;
    r->keys[0] = keys ? keys[0] : 0;
    r->ext[0] = ptrs ? (char*)ptrs[0] : nullptr;
    r->bytes_alg = n * es;
  } else {
    Analysis an;
    std::string err;
    salt_status st = analyse(prog, nprog, nkeys, nscal, &an, &err);
    if (st != SALT_OK) {
      delete r;
      return fail(st, err);
    }
    if (an.used_scals && !scalars) {
      delete r;
      return fail(SALT_ERR_ARG, "scalars is NULL");
    }
    // Scalar subexpressions of by-value scalars are computed here, once
    // (a served request takes no device scalars).
    Hoisted h;
    double sc2[kMaxScals] = {};
    if (an.scalar_nodes) {
      st = hoist_scalars(prog, nprog, nscal, &h, &err);
      if (st != SALT_OK) {
        delete r;
        return fail(st, err);
      }
      for (int k = 0; k < nscal; ++k) sc2[k] = scalars[k];
      for (int j = 0; j < h.nhoist; ++j)
        sc2[nscal + j] = dtype == SALT_F32 ? host_scalar_value_f32(prog, h, j, sc2)
                                           : host_scalar_value_f64(prog, h, j, sc2);
      prog = h.prog;
      nprog = h.nprog;
      nscal = h.nscal;
      scalars = sc2;
    }
    Canonical c;
    canonicalise(prog, nprog, &c);
    const int shape = find_shape(c);
    if (shape < 0 || shape >= NUM_BATCH_SHAPES || c.nvec > kBatchOps || c.nscal > 2 || c.nred > kBatchPartials) {
      delete r;
      return fail(SALT_ERR_PROGRAM, "program has no compiled instantiation the server can batch");
    }
    r->kind = shape;
    r->nvec = c.nvec;
    r->load_mask = c.load_mask;
    r->nred = c.nred;
    for (int k = 0; k < c.nvec; ++k) {
      r->user_of[k] = c.vec_user[k];
      r->ext[k] = ptrs ? (char*)ptrs[c.vec_user[k]] : nullptr;
      if (!r->ext[k] && !keys) {
        delete r;
        return fail(SALT_ERR_ARG, "an operand has neither a pointer nor a key");
      }
      r->keys[k] = r->ext[k] ? 0 : keys[c.vec_user[k]];
    }
    for (int k = 0; k < c.nscal; ++k) {
      const double v = scalars[c.scal_user[k]];
      r->sc[k] = dtype == SALT_F32 ? (double)(float)v : v;
    }
    r->bytes_alg = (int64_t)(__builtin_popcount(c.load_mask) + __builtin_popcount(c.store_mask)) * es * n;
  }
  r->vec_bytes = round_up((size_t)std::max<int64_t>(n, 1) * es);
  int owned = 0;
  for (int k = 0; k < r->nvec; ++k) owned += r->ext[k] == nullptr;
  if ((int64_t)(r->vec_bytes * owned) > s->cfg.budget_bytes) {
    delete r;
    return fail(SALT_ERR_BUDGET, "request needs more device memory than the whole budget");
  }
  r->t_submit = t_submit;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return fail(SALT_ERR_ARG, s->sched_error.empty() ? "server is stopping" : s->sched_error);
  }
  r->id = s->next_id++;
  s->reqs[r->id] = r;
  s->waiting.push_back(r);
  *id_out = r->id;
  s->cv.notify_all();
  return SALT_OK;
}

void release_locked(salt_server* s, Request* r) {
  if (r->resident) {
    arena_give(s, r);
    r->resident = false;
    --s->resident;
  }
  s->reqs.erase(r->id);
  delete r;
  s->cv.notify_all();
}

}  // namespace

namespace salt {
unsigned serve_polls(int64_t set) {
  if (set >= 0) g_serve_polls.store((unsigned)set);
  return g_serve_polls.load();
}
}  // namespace salt

extern "C" {

salt_status salt_serve_default_config(salt_serve_config* cfg) {
  if (!cfg) return fail(SALT_ERR_ARG, "cfg is NULL");
  cfg->budget_bytes = (int64_t)8 << 30;
  cfg->max_requests = 4096;
  cfg->max_batch = 256;
  cfg->streams = 2;
  cfg->tile_bytes = 64 * 1024;
  cfg->unroll = 2;
  cfg->block = 256;
  cfg->max_n = (int64_t)1 << 24;
  cfg->persistent = 0;
  cfg->idle_us = 10000;
  return SALT_OK;
}

salt_status salt_serve_start(salt_server** out, const salt_serve_config* cfg) {
  if (!out || !cfg) return fail(SALT_ERR_ARG, "out or cfg is NULL");
  if (cfg->budget_bytes < (1 << 20) || cfg->max_requests < 1 || cfg->max_batch < 1 || cfg->max_batch > 65536 ||
      cfg->streams < 1 || cfg->streams > 8 || cfg->tile_bytes < 1024 || cfg->tile_bytes % 256 ||
      (cfg->unroll != 1 && cfg->unroll != 2 && cfg->unroll != 4) ||
      (cfg->block != 64 && cfg->block != 128 && cfg->block != 256) || cfg->max_n < 1 ||
      (cfg->persistent != 0 && cfg->persistent != 1) || cfg->idle_us < 1 || cfg->idle_us > 10000000)
    return fail(SALT_ERR_ARG, "invalid server configuration");
  int dev = 0, sms = 0;
  salt_status st = current_device(&dev, &sms);
  if (st != SALT_OK) return st;
  salt_server* s = new salt_server();
  s->cfg = *cfg;
  s->device = dev;
  s->sms = sms;
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)kernel_for(cfg->unroll), cfg->block, 0);
  s->grid = sms * std::max(bps, 1);
  s->items_cap = (int64_t)cfg->max_batch * kBatchOps;
  const int64_t per_req_tiles = (cfg->max_n * 8 + cfg->tile_bytes - 1) / cfg->tile_bytes;
  s->tiles_cap = std::max<int64_t>((int64_t)cfg->max_batch * 4, per_req_tiles * 4);
  cudaError_t e = cudaMalloc(&s->arena_base, (size_t)cfg->budget_bytes);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaMalloc(arena)");
  }
  s->arena.init((size_t)cfg->budget_bytes);
  s->slots.resize(cfg->persistent ? 0 : (size_t)cfg->streams);
  size_t off_items[2], off_counters[2], off_partials;
  const size_t dbytes = slot_device_bytes(s, off_items, off_counters, &off_partials);
  for (Slot& slot : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&slot.d_mem, dbytes);
    slot.table_bytes = off_counters[0];
    if (e == cudaSuccess) e = cudaHostAlloc(&slot.h_mem, slot.table_bytes, cudaHostAllocDefault);
    if (e == cudaSuccess)
      e = cudaHostAlloc(&slot.h_red, sizeof(double) * kBatchPartials * cfg->max_batch, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&slot.h_red_dev, slot.h_red, 0);
    if (e != cudaSuccess) break;
    slot.compute_items.resize((size_t)s->cfg.max_batch);
    for (int t = 0; t < 2; ++t) slot.d_counters[t] = (unsigned*)(slot.d_mem + off_counters[t]);
    slot.d_partials = (double*)(slot.d_mem + off_partials);
    // the counters start at zero; every launch leaves them at zero
    e = cudaMemset(slot.d_mem + off_counters[0], 0, off_partials - off_counters[0]);
    for (int f = 0; f < 2 && e == cudaSuccess; ++f) e = build_step_graph(s, slot, f == 1, &slot.g[f]);
  }
  if (e != cudaSuccess) {
    for (Slot& slot : s->slots) {
      if (slot.d_mem) cudaFree(slot.d_mem);
      if (slot.h_mem) cudaFreeHost(slot.h_mem);
      if (slot.h_red) cudaFreeHost(slot.h_red);
      for (Slot::StepGraph& sg : slot.g) {
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        if (sg.graph) cudaGraphDestroy(sg.graph);
      }
      if (slot.done) cudaEventDestroy(slot.done);
      if (slot.stream) cudaStreamDestroy(slot.stream);
    }
    cudaFree(s->arena_base);
    delete s;
    return cuda_fail(e, "server resources");
  }
  if (cfg->persistent) {
    st = persist_init(s);
    if (st != SALT_OK) {
      cudaFree(s->arena_base);
      delete s;
      return st;
    }
  }
  s->sched = std::thread(cfg->persistent ? scheduler_persist : scheduler, s);
  *out = s;
  return SALT_OK;
}

salt_status salt_serve_submit(salt_server* s, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                              const uint64_t* keys, int32_t nkeys, const double* scalars, int32_t nscal,
                              int64_t* request_id) {
  if (!s || !request_id) return fail(SALT_ERR_ARG, "server or request_id is NULL");
  return submit_impl(s, prog, nprog, dtype, n, nullptr, keys, nkeys, scalars, nscal, now_us(), request_id);
}

salt_status salt_serve_submit_ex(salt_server* s, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                                 const void* const* ptrs, const uint64_t* keys, int32_t nops,
                                 const double* scalars, int32_t nscal, int64_t* request_id) {
  if (!s || !request_id) return fail(SALT_ERR_ARG, "server or request_id is NULL");
  return submit_impl(s, prog, nprog, dtype, n, ptrs, keys, nops, scalars, nscal, now_us(), request_id);
}

salt_status salt_serve_poll(salt_server* s, int64_t id, int32_t* state, double* latency_us, double* red) {
  if (!s) return fail(SALT_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(SALT_ERR_NOTFOUND, "unknown request id");
  const Request* r = it->second;
  if (state) *state = r->state;
  if (r->state == RS_DONE) {
    if (latency_us) *latency_us = r->t_done - r->t_submit;
    if (red)
      for (int j = 0; j < r->nred; ++j) red[j] = r->red[j];
  }
  return SALT_OK;
}

salt_status salt_serve_wait(salt_server* s, int64_t id, int64_t timeout_us) {
  if (!s) return fail(SALT_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  for (;;) {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(SALT_ERR_NOTFOUND, "unknown request id");
    if (it->second->state == RS_DONE) return SALT_OK;
    if (s->stop && !s->sched_error.empty()) return fail(SALT_ERR_CUDA, s->sched_error);
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = s->reqs.find(id);
      if (it != s->reqs.end() && it->second->state == RS_DONE) return SALT_OK;
      return fail(SALT_ERR_TIMEOUT, "request not complete within the timeout");
    }
  }
}

salt_status salt_serve_read(salt_server* s, int64_t id, int32_t operand, void* host_dst, int64_t bytes) {
  if (!s || !host_dst) return fail(SALT_ERR_ARG, "server or host_dst is NULL");
  char* src = nullptr;
  int64_t n = 0, es = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(SALT_ERR_NOTFOUND, "unknown request id");
    Request* r = it->second;
    if (r->state != RS_DONE) return fail(SALT_ERR_ARG, "request is not complete");
    int k = -1;
    for (int j = 0; j < r->nvec; ++j)
      if ((r->kind == kKindNrm2 ? 0 : r->user_of[j]) == operand) k = j;
    if (k < 0) return fail(SALT_ERR_ARG, "request has no such operand");
    es = r->dtype == SALT_F32 ? 4 : 8;
    n = r->n;
    if (bytes < n * es) return fail(SALT_ERR_ARG, "host buffer too small");
    src = operand_ptr(s, r, k);
  }
  if (n == 0) return SALT_OK;
  cudaError_t e = cudaMemcpy(host_dst, src, (size_t)(n * es), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SALT_OK : cuda_fail(e, "cudaMemcpy(read)");
}

salt_status salt_serve_release(salt_server* s, int64_t id) {
  if (!s) return fail(SALT_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(SALT_ERR_NOTFOUND, "unknown request id");
  Request* r = it->second;
  if (r->state == RS_RUNNING) return fail(SALT_ERR_ARG, "request is running; wait for it first");
  if (r->state == RS_WAITING) {
    auto w = std::find(s->waiting.begin(), s->waiting.end(), r);
    if (w != s->waiting.end()) s->waiting.erase(w);
    auto p = std::find(s->pending.begin(), s->pending.end(), r);
    if (p != s->pending.end()) s->pending.erase(p);
  }
  release_locked(s, r);
  return SALT_OK;
}

salt_status salt_serve_stats(salt_server* s, int64_t* completed, int64_t* steps, int64_t* bytes,
                             int64_t* resident_bytes, int32_t* waiting) {
  if (!s) return fail(SALT_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->n_done.load();
  if (steps) *steps = s->n_steps.load();
  if (bytes) *bytes = s->bytes_done.load();
  if (resident_bytes) *resident_bytes = (int64_t)s->arena.used();
  if (waiting) *waiting = (int32_t)(s->waiting.size() + s->pending.size());
  return SALT_OK;
}

salt_status salt_serve_launches(salt_server* s, int64_t* launches, int32_t* live) {
  if (!s) return fail(SALT_ERR_ARG, "server is NULL");
  if (launches) *launches = s->ps.launches.load();
  if (live) *live = s->ps.live.load() ? 1 : 0;
  return SALT_OK;
}

salt_status salt_serve_stop(salt_server* s) {
  if (!s) return SALT_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->sched.joinable()) s->sched.join();
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  if (s->ps.on) persist_free(s);
  for (Slot& slot : s->slots) {
    if (slot.stream) cudaStreamSynchronize(slot.stream);
    if (slot.d_mem) cudaFree(slot.d_mem);
    if (slot.h_mem) cudaFreeHost(slot.h_mem);
    if (slot.h_red) cudaFreeHost(slot.h_red);
    for (Slot::StepGraph& sg : slot.g) {
      if (sg.exec) cudaGraphExecDestroy(sg.exec);
      if (sg.graph) cudaGraphDestroy(sg.graph);
    }
    if (slot.done) cudaEventDestroy(slot.done);
    if (slot.stream) cudaStreamDestroy(slot.stream);
  }
  cudaFree(s->arena_base);
  cudaSetDevice(cur);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return SALT_OK;
}

}  // extern "C"

namespace {

// Standard served shapes of the load generator and, per shape, the operands
// it stores (those never come from a caller's store).
const salt_insn kReplayProgs[4][12] = {
    {{SALT_OP_VEC, 0}, {SALT_OP_VEC, 1}, {SALT_OP_VEC, 2}, {SALT_OP_SUB, 0}, {SALT_OP_ADD, 0}, {SALT_OP_STORE, 3}},
    {{SALT_OP_SCAL, 0}, {SALT_OP_VEC, 0}, {SALT_OP_SMUL, 0}, {SALT_OP_SCAL, 1}, {SALT_OP_VEC, 1},
     {SALT_OP_SMUL, 0}, {SALT_OP_ADD, 0}, {SALT_OP_STORE, 1}},
    {{SALT_OP_SCAL, 0}, {SALT_OP_VEC, 0}, {SALT_OP_SMUL, 0}, {SALT_OP_SCAL, 1}, {SALT_OP_VEC, 1},
     {SALT_OP_SMUL, 0}, {SALT_OP_ADD, 0}, {SALT_OP_VEC, 2}, {SALT_OP_VEC, 3}, {SALT_OP_MUL, 0},
     {SALT_OP_SUB, 0}, {SALT_OP_STORE, 4}},
    {{SALT_OP_VEC, 0}, {SALT_OP_VEC, 1}, {SALT_OP_DOT, 0}}};
const int32_t kReplayLen[4] = {6, 8, 12, 3};
const int32_t kReplayVecs[5] = {4, 2, 5, 2, 1};
const int32_t kReplayStored[5] = {3, 1, 4, -1, -1};  // stored operand per shape, or -1

struct ReplayStore {
  const void* const* vec[2] = {nullptr, nullptr};  // [F32, F64] store vectors
  int32_t count[2] = {0, 0};
  int64_t len[2] = {0, 0};
};

salt_status replay_impl(salt_server* s, int32_t count, const double* arrival_us, const int32_t* shape,
                        const int32_t* dtype, const int64_t* n, uint64_t seed, const ReplayStore* store,
                        double* latency_us, double* red_first, double* wall_us) {
  if (!s || count < 0 || (count > 0 && (!arrival_us || !shape || !dtype || !n || !latency_us)))
    return fail(SALT_ERR_ARG, "bad replay arguments");
  const double sc[2] = {1.5, -0.25};
  std::vector<int64_t> ids((size_t)count, 0);
  std::unordered_map<int64_t, int32_t> index_of;
  const double t0 = now_us();
  int32_t next = 0, done = 0;
  double last_done = t0;
  while (done < count) {
    const double t = now_us() - t0;
    while (next < count && arrival_us[next] <= t) {
      const int sh = shape[next];
      if (sh < 0 || sh > 4) return fail(SALT_ERR_ARG, "shape index outside 0..4");
      uint64_t keys[kBatchOps];
      const void* ptrs[kBatchOps] = {nullptr, nullptr, nullptr, nullptr, nullptr};
      for (int k = 0; k < kReplayVecs[sh]; ++k) {
        keys[k] = vector_key(seed, (uint64_t)next, (uint64_t)k);
        if (store && k != kReplayStored[sh]) {
          const int t2 = dtype[next] == SALT_F64 ? 1 : 0;
          const int64_t len = store->len[t2], nn = n[next];
          if (store->count[t2] < 1 || nn > len) return fail(SALT_ERR_ARG, "store has no vector long enough");
          ptrs[k] = (const char*)store->vec[t2][store_vector(next, k, store->count[t2])] +
                    store_offset(seed, (uint64_t)next, (uint64_t)k, nn, len, dtype[next] == SALT_F64 ? 4 : 8) *
                        (dtype[next] == SALT_F64 ? 8 : 4);
        }
      }
      int64_t id = 0;
      salt_status st = submit_impl(s, sh == 4 ? nullptr : kReplayProgs[sh], sh == 4 ? 0 : kReplayLen[sh],
                                   dtype[next], n[next], store ? ptrs : nullptr, keys, kReplayVecs[sh], sc, 2,
                                   t0 + arrival_us[next], &id);
      if (st != SALT_OK) return st;
      ids[(size_t)next] = id;
      index_of[id] = next;
      ++next;
    }
    std::vector<int64_t> finished;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && !s->sched_error.empty()) return fail(SALT_ERR_CUDA, s->sched_error);
      if (s->completed.empty()) {
        // Sleep only well ahead of the next arrival (a timed wait may
        // oversleep by the timer slack, tens of microseconds); close to it,
        // or while requests are in flight, yield and look again.
        const double wait = next < count ? std::max(0.0, arrival_us[next] - (now_us() - t0)) : 200.0;
        if (wait > 150.0) {
          s->cv.wait_for(lk, std::chrono::microseconds((int64_t)std::min(wait - 100.0, 200.0)));
        } else {
          lk.unlock();
          std::this_thread::yield();
          lk.lock();
        }
      }
      while (!s->completed.empty()) {
        finished.push_back(s->completed.front());
        s->completed.pop_front();
      }
      for (int64_t id : finished) {
        auto it = index_of.find(id);
        auto rq = s->reqs.find(id);
        if (it == index_of.end() || rq == s->reqs.end()) continue;  // not ours
        Request* r = rq->second;
        latency_us[it->second] = r->t_done - r->t_submit;
        if (red_first) red_first[it->second] = r->nred > 0 ? r->red[0] : 0.0;
        last_done = std::max(last_done, r->t_done);
        release_locked(s, r);
        index_of.erase(it);
        ++done;
      }
    }
  }
  if (wall_us) *wall_us = last_done - t0;
  return SALT_OK;
}

}  // namespace

extern "C" {

salt_status salt_serve_replay(salt_server* s, int32_t count, const double* arrival_us, const int32_t* shape,
                              const int32_t* dtype, const int64_t* n, uint64_t seed, double* latency_us,
                              double* red_first, double* wall_us) {
  return replay_impl(s, count, arrival_us, shape, dtype, n, seed, nullptr, latency_us, red_first, wall_us);
}

salt_status salt_serve_replay_store(salt_server* s, int32_t count, const double* arrival_us, const int32_t* shape,
                                    const int32_t* dtype, const int64_t* n, uint64_t seed,
                                    const void* const* store_f32, int32_t nstore_f32, int64_t len_f32,
                                    const void* const* store_f64, int32_t nstore_f64, int64_t len_f64,
                                    double* latency_us, double* red_first, double* wall_us) {
  if (nstore_f32 < 0 || nstore_f64 < 0 || (nstore_f32 > 0 && !store_f32) || (nstore_f64 > 0 && !store_f64))
    return fail(SALT_ERR_ARG, "bad store");
  for (int i = 0; i < nstore_f32; ++i)
    if (!store_f32[i] || (uintptr_t)store_f32[i] % 16) return fail(SALT_ERR_ALIGN, "store vectors must be 16-byte aligned");
  for (int i = 0; i < nstore_f64; ++i)
    if (!store_f64[i] || (uintptr_t)store_f64[i] % 16) return fail(SALT_ERR_ALIGN, "store vectors must be 16-byte aligned");
  ReplayStore st;
  st.vec[0] = store_f32;
  st.vec[1] = store_f64;
  st.count[0] = nstore_f32;
  st.count[1] = nstore_f64;
  st.len[0] = len_f32;
  st.len[1] = len_f64;
  return replay_impl(s, count, arrival_us, shape, dtype, n, seed, &st, latency_us, red_first, wall_us);
}

}  // extern "C"
