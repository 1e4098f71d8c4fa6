// Batch API (include/salt.h, salt_batch_*): item table, validation, one
// persistent launch captured in a CUDA graph, the plain per-call path for
// comparison, and an autotuner over the launch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/salt.h"
#include "batch.cuh"
#include "internal.h"
#include "registry.h"

using namespace salt;

namespace {

struct HostItem {
  std::vector<salt_insn> prog;  // empty for nrm2 items
  std::vector<void*> vecs;      // user operands (program order)
  std::vector<double> scalars;
  int32_t dtype;
  int64_t n;
  int32_t nred;
  BatchItem dev;                // device descriptor (tile fields filled at build)
  uint32_t store_mask_c;        // canonical operands that are written
};

using KernelFn = void (*)(const BatchParams);
KernelFn kernel_for(int unroll) {
  switch (unroll) {
    case 1: return &batch_kernel<1>;
    case 2: return &batch_kernel<2>;
    default: return &batch_kernel<4>;
  }
}

constexpr size_t kHeaderBytes = 256;

}  // namespace

struct salt_batch {
  int32_t capacity = 0;
  std::vector<HostItem> items;
  int32_t nresults = 0;
  // launch shape
  int32_t unroll = 2, block = 256, blocks_per_sm = 0;
  int64_t tile_bytes = 64 * 1024;
  int32_t vec_bytes = 32;  // widest access for 32-byte aligned FP32 items (16 or 32)
  // device state
  int device = -1;
  void* dmem = nullptr;           // header | items | counter+tickets | partials
  size_t dmem_bytes = 0;
  int64_t tiles_capacity = 0;
  BatchHeader* d_hdr = nullptr;
  BatchItem* d_items = nullptr;
  unsigned* d_counters = nullptr;  // [0] tile counter, [1] finished blocks, [2..capacity+1] tickets
  double* d_partials = nullptr;
  int64_t total_tiles = 0;
  bool dirty = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* graph_red_out = nullptr;
  int graph_grid = 0;
};

namespace {

salt_status fail(salt_status st, const std::string& m) { return report_error(st, m); }
salt_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SALT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void drop_graph(salt_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_red_out = nullptr;
}

int64_t tile_elems_of(const salt_batch* b, int dtype) { return b->tile_bytes / (dtype == SALT_F32 ? 4 : 8); }

// Items may not write memory that another item of the same batch reads or
// writes: their tiles run in any order.
salt_status check_cross_item_overlap(const salt_batch* b) {
  struct Range {
    uintptr_t lo, hi;
    int item;
    bool write;
  };
  std::vector<Range> rs;
  for (size_t i = 0; i < b->items.size(); ++i) {
    const HostItem& it = b->items[i];
    const uintptr_t bytes = (uintptr_t)it.n * (it.dtype == SALT_F32 ? 4 : 8);
    if (bytes == 0) continue;
    for (int k = 0; k < kBatchOps; ++k) {
      if (!it.dev.v[k]) continue;
      const uintptr_t lo = (uintptr_t)it.dev.v[k];
      rs.push_back({lo, lo + bytes, (int)i, ((it.store_mask_c >> k) & 1u) != 0});
    }
  }
  std::sort(rs.begin(), rs.end(), [](const Range& a, const Range& c) { return a.lo < c.lo; });
  // sweep: compare each range with the active ranges that overlap it
  std::vector<Range> active;
  for (const Range& r : rs) {
    active.erase(std::remove_if(active.begin(), active.end(), [&](const Range& a) { return a.hi <= r.lo; }),
                 active.end());
    for (const Range& a : active) {
      if (a.item != r.item && (a.write || r.write)) {
        char buf[160];
        snprintf(buf, sizeof buf, "items %d and %d overlap in memory and one of them writes it", a.item, r.item);
        return fail(SALT_ERR_ALIAS, buf);
      }
    }
    active.push_back(r);
  }
  return SALT_OK;
}

// Lays items out in tiles, (re)allocates device buffers, uploads the table.
salt_status rebuild(salt_batch* b, cudaStream_t s) {
  salt_status st = check_cross_item_overlap(b);
  if (st != SALT_OK) return st;
  int dev = 0, sms = 0;
  st = current_device(&dev, &sms);
  if (st != SALT_OK) return st;
  // earlier launches of this batch may still read the table
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  drop_graph(b);
  int64_t tile = 0;
  for (HostItem& it : b->items) {
    const int64_t te = tile_elems_of(b, it.dtype);
    const int64_t nt = it.n > 0 ? (it.n + te - 1) / te : 1;
    it.dev.tile_begin = tile;
    it.dev.ntiles = (int32_t)nt;
    tile += nt;
  }
  b->total_tiles = tile;
  if (tile >= (int64_t)1 << 31) return fail(SALT_ERR_BUDGET, "batch has more than 2^31 tiles; raise tile_bytes");
  if (b->dmem == nullptr || b->device != dev || tile > b->tiles_capacity) {
    if (b->dmem) cudaFree(b->dmem);
    b->dmem = nullptr;
    const int64_t tiles_cap = std::max<int64_t>(tile, 1024);
    const size_t items_bytes = ((sizeof(BatchItem) * (size_t)b->capacity + 255) / 256) * 256;
    const size_t counters_bytes = ((sizeof(unsigned) * (size_t)(b->capacity + 2) + 255) / 256) * 256;
    const size_t partial_bytes = sizeof(double) * kBatchPartials * (size_t)tiles_cap;
    const size_t total = kHeaderBytes + items_bytes + counters_bytes + partial_bytes;
    e = cudaMalloc(&b->dmem, total);
    if (e != cudaSuccess) {
      b->dmem = nullptr;
      return cuda_fail(e, "cudaMalloc(batch)");
    }
    char* base = (char*)b->dmem;
    b->d_hdr = (BatchHeader*)base;
    b->d_items = (BatchItem*)(base + kHeaderBytes);
    b->d_counters = (unsigned*)(base + kHeaderBytes + items_bytes);
    b->d_partials = (double*)(base + kHeaderBytes + items_bytes + counters_bytes);
    b->dmem_bytes = total;
    b->tiles_capacity = tiles_cap;
    b->device = dev;
    e = cudaMemset(b->d_counters, 0, counters_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(batch)");
  }
  BatchHeader h{};
  h.nitems = (int32_t)b->items.size();
  h.total_tiles = b->total_tiles;
  h.tile_bytes = b->tile_bytes;
  h.narrow = b->vec_bytes == 16 ? 1 : 0;
  std::vector<BatchItem> table(b->items.size());
  for (size_t i = 0; i < b->items.size(); ++i) table[i] = b->items[i].dev;
  e = cudaMemcpy(b->d_hdr, &h, sizeof h, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !table.empty())
    e = cudaMemcpy(b->d_items, table.data(), sizeof(BatchItem) * table.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(batch table)");
  b->dirty = false;
  return SALT_OK;
}

int occupancy(KernelFn k, int block) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k, block, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb < 1 ? 1 : nb;
}

salt_status build_graph(salt_batch* b, double* red_out) {
  drop_graph(b);
  int dev = 0, sms = 0;
  salt_status st = current_device(&dev, &sms);
  if (st != SALT_OK) return st;
  KernelFn k = kernel_for(b->unroll);
  int bps = b->blocks_per_sm > 0 ? b->blocks_per_sm : occupancy(k, b->block);
  int64_t grid = (int64_t)sms * bps;
  if (grid > b->total_tiles) grid = b->total_tiles;
  if (grid < 1) grid = 1;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  cudaMemsetParams mp{};
  mp.dst = b->d_counters;
  mp.value = 0;
  mp.elementSize = sizeof(unsigned);
  mp.width = (size_t)b->items.size() + 2;
  mp.height = 1;
  mp.pitch = 0;
  cudaGraphNode_t mnode = nullptr, knode = nullptr;
  e = cudaGraphAddMemsetNode(&mnode, g, nullptr, 0, &mp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphAddMemsetNode");
  }
  BatchParams p{b->d_hdr, b->d_items, b->d_counters, b->d_counters + 1, b->d_counters + 2, b->d_partials, red_out};
  void* args[] = {&p};
  cudaKernelNodeParams kp{};
  kp.func = (void*)k;
  kp.gridDim = dim3((unsigned)grid);
  kp.blockDim = dim3((unsigned)b->block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  e = cudaGraphAddKernelNode(&knode, g, &mnode, 1, &kp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphAddKernelNode");
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  b->graph = g;
  b->exec = x;
  b->graph_red_out = red_out;
  b->graph_grid = (int)grid;
  return SALT_OK;
}

salt_status launch(salt_batch* b, double* red_out, cudaStream_t s) {
  if (b->items.empty()) return SALT_OK;
  if (b->nresults > 0 && !red_out) return fail(SALT_ERR_ARG, "red_out is NULL but the batch has reductions");
  if (red_out && ((uintptr_t)red_out % 8)) return fail(SALT_ERR_ALIGN, "red_out must be 8-byte aligned");
  salt_status st;
  if (b->dirty) {
    st = rebuild(b, s);
    if (st != SALT_OK) return st;
  }
  if (!b->exec || b->graph_red_out != red_out) {
    st = build_graph(b, red_out);
    if (st != SALT_OK) return st;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  count_launch();
  return e == cudaSuccess ? SALT_OK : cuda_fail(e, "cudaGraphLaunch");
}

}  // namespace

extern "C" {

salt_status salt_batch_create(salt_batch** out, int32_t capacity) {
  if (!out) return fail(SALT_ERR_ARG, "out is NULL");
  if (capacity < 1 || capacity > (1 << 20)) return fail(SALT_ERR_ARG, "capacity outside 1..2^20");
  salt_batch* b = new salt_batch();
  b->capacity = capacity;
  b->items.reserve((size_t)capacity);
  *out = b;
  return SALT_OK;
}

salt_status salt_batch_destroy(salt_batch* b) {
  if (!b) return SALT_OK;
  drop_graph(b);
  if (b->dmem) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (b->device >= 0) cudaSetDevice(b->device);
    cudaFree(b->dmem);
    cudaSetDevice(cur);
  }
  delete b;
  return SALT_OK;
}

salt_status salt_batch_add(salt_batch* b, const salt_insn* prog, int32_t nprog, int32_t dtype, int64_t n,
                           void* const* vecs, int32_t nvecs, const double* scalars, int32_t nscal,
                           int32_t* red_index_out) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if ((int32_t)b->items.size() >= b->capacity) return fail(SALT_ERR_BUDGET, "batch is full");
  EvalArgs a{prog, nprog, dtype, n, vecs, nvecs, scalars, nscal, nullptr, nullptr};
  Analysis an;
  // validate as a salt_eval call (result buffer supplied at launch)
  double dummy_red[kMaxReds];
  a.red_out = dummy_red;
  salt_status st = validate_eval(a, &an);
  if (st != SALT_OK) return st;
  // Scalar subexpressions (by-value scalars only: a batch takes no device
  // scalars) are computed here; the item carries the hoisted program.
  Hoisted h;
  double sc2[kMaxScals] = {};
  if (an.scalar_nodes) {
    std::string err;
    st = hoist_scalars(prog, nprog, nscal, &h, &err);
    if (st != SALT_OK) return fail(st, err);
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
  if (shape < 0 || shape >= NUM_BATCH_SHAPES)
    return fail(SALT_ERR_PROGRAM, "program has no instantiation in the batch kernel, so it cannot be batched");
  if (c.nvec > kBatchOps || c.nscal > 2 || c.nred > kBatchPartials)
    return fail(SALT_ERR_PROGRAM, "program exceeds the batch item limits");
  for (int k = 0; k < c.nvec && n > 0; ++k) {
    if (!vecs[c.vec_user[k]]) return fail(SALT_ERR_ARG, "operand is NULL");
    if ((uintptr_t)vecs[c.vec_user[k]] % 16) return fail(SALT_ERR_ALIGN, "batch operands must be 16-byte aligned");
  }
  HostItem it;
  it.prog.assign(prog, prog + nprog);
  it.vecs.assign(vecs, vecs + nvecs);
  it.scalars.assign(scalars ? scalars : dummy_red, scalars ? scalars + nscal : dummy_red);
  it.dtype = dtype;
  it.n = n;
  it.nred = c.nred;
  it.store_mask_c = c.store_mask;
  memset(&it.dev, 0, sizeof it.dev);
  it.dev.kind = shape;
  it.dev.dtype = dtype == SALT_F32 ? DT_F32 : DT_F64;
  it.dev.n = n;
  it.dev.red_index = c.nred > 0 ? b->nresults : -1;
  for (int k = 0; k < c.nvec; ++k) it.dev.v[k] = vecs[c.vec_user[k]];
  for (int k = 0; k < c.nscal; ++k) {
    const double s = scalars[c.scal_user[k]];
    it.dev.sc[k] = dtype == SALT_F32 ? (double)(float)s : s;
  }
  if (red_index_out) *red_index_out = it.dev.red_index;
  b->nresults += c.nred;
  b->items.push_back(std::move(it));
  b->dirty = true;
  return SALT_OK;
}

salt_status salt_batch_add_nrm2(salt_batch* b, int32_t dtype, int64_t n, const void* x, int32_t* red_index_out) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if ((int32_t)b->items.size() >= b->capacity) return fail(SALT_ERR_BUDGET, "batch is full");
  if (dtype != SALT_F32 && dtype != SALT_F64) return fail(SALT_ERR_DTYPE, "dtype must be SALT_F32 or SALT_F64");
  if (n < 0) return fail(SALT_ERR_ARG, "n must be >= 0");
  if (n > 0 && !x) return fail(SALT_ERR_ARG, "x is NULL");
  if ((uintptr_t)x % 16) return fail(SALT_ERR_ALIGN, "x must be 16-byte aligned");
  HostItem it;
  it.vecs.assign(1, const_cast<void*>(x));
  it.dtype = dtype;
  it.n = n;
  it.nred = 1;
  it.store_mask_c = 0;
  memset(&it.dev, 0, sizeof it.dev);
  it.dev.kind = kKindNrm2;
  it.dev.dtype = dtype == SALT_F32 ? DT_F32 : DT_F64;
  it.dev.n = n;
  it.dev.red_index = b->nresults;
  it.dev.v[0] = const_cast<void*>(x);
  if (red_index_out) *red_index_out = it.dev.red_index;
  b->nresults += 1;
  b->items.push_back(std::move(it));
  b->dirty = true;
  return SALT_OK;
}

salt_status salt_batch_clear(salt_batch* b) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  b->items.clear();
  b->nresults = 0;
  b->dirty = true;
  return SALT_OK;
}

salt_status salt_batch_info(const salt_batch* b, int32_t* nitems, int32_t* nresults, int64_t* bytes) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if (nitems) *nitems = (int32_t)b->items.size();
  if (nresults) *nresults = b->nresults;
  if (bytes) {
    int64_t tot = 0;
    for (const HostItem& it : b->items) {
      const int64_t es = it.dtype == SALT_F32 ? 4 : 8;
      int ops = 1;
      if (it.dev.kind != kKindNrm2) {
        Canonical c;
        canonicalise(it.prog.data(), (int)it.prog.size(), &c);
        ops = __builtin_popcount(c.load_mask) + __builtin_popcount(c.store_mask);
      }
      tot += ops * es * it.n;
    }
    *bytes = tot;
  }
  return SALT_OK;
}

salt_status salt_batch_set_config(salt_batch* b, int32_t unroll, int32_t block, int32_t blocks_per_sm,
                                  int64_t tile_bytes) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if ((unroll != 1 && unroll != 2 && unroll != 4) || (block != 64 && block != 128 && block != 256) ||
      blocks_per_sm < 0 || blocks_per_sm > 32 || tile_bytes < 1024 || tile_bytes % 256 ||
      tile_bytes > ((int64_t)1 << 26))
    return fail(SALT_ERR_ARG, "invalid batch configuration");
  if (tile_bytes != b->tile_bytes) b->dirty = true;
  b->unroll = unroll;
  b->block = block;
  b->blocks_per_sm = blocks_per_sm;
  b->tile_bytes = tile_bytes;
  drop_graph(b);
  return SALT_OK;
}

salt_status salt_batch_get_config(const salt_batch* b, int32_t* unroll, int32_t* block, int32_t* blocks_per_sm,
                                  int64_t* tile_bytes) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if (unroll) *unroll = b->unroll;
  if (block) *block = b->block;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  if (tile_bytes) *tile_bytes = b->tile_bytes;
  return SALT_OK;
}

salt_status salt_batch_launch(salt_batch* b, double* red_out, void* stream) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  return launch(b, red_out, (cudaStream_t)stream);
}

salt_status salt_batch_launch_plain(salt_batch* b, double* red_out, void* stream) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if (b->nresults > 0 && !red_out) return fail(SALT_ERR_ARG, "red_out is NULL but the batch has reductions");
  const cudaStream_t s = (cudaStream_t)stream;
  for (HostItem& it : b->items) {
    salt_status st;
    if (it.dev.kind == kKindNrm2) {
      st = nrm2_impl(it.dtype, it.n, it.vecs[0], red_out + it.dev.red_index, SALT_DEFAULT, s);
    } else {
      EvalArgs a{it.prog.data(), (int)it.prog.size(), it.dtype, it.n, it.vecs.data(), (int)it.vecs.size(),
                 it.scalars.data(), (int)it.scalars.size(), it.nred > 0 ? red_out + it.dev.red_index : nullptr, s};
      st = eval_impl(a);
    }
    if (st != SALT_OK) return st;
  }
  return SALT_OK;
}

salt_status salt_batch_set_vec_bytes(salt_batch* b, int32_t vec_bytes) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if (vec_bytes != 16 && vec_bytes != 32) return fail(SALT_ERR_ARG, "vec_bytes must be 16 or 32");
  if (vec_bytes != b->vec_bytes) {
    b->vec_bytes = vec_bytes;
    b->dirty = true;  // the header carries it
    drop_graph(b);
  }
  return SALT_OK;
}

salt_status salt_batch_get_vec_bytes(const salt_batch* b, int32_t* vec_bytes) {
  if (!b || !vec_bytes) return fail(SALT_ERR_ARG, "batch or vec_bytes is NULL");
  *vec_bytes = b->vec_bytes;
  return SALT_OK;
}

salt_status salt_batch_autotune(salt_batch* b, double* red_out, int32_t reps, double* best_ms, void* stream) {
  if (!b) return fail(SALT_ERR_ARG, "batch is NULL");
  if (reps < 1) return fail(SALT_ERR_ARG, "reps must be >= 1");
  const cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(SALT_ERR_CUDA, "cudaEventCreate");
  const int32_t unrolls[] = {1, 2, 4};
  const int32_t blocks[] = {128, 256};
  const int64_t tiles[] = {16 * 1024, 32 * 1024, 64 * 1024, 128 * 1024};
  // the vector width matters only for FP32 items whose operands are all
  // 32-byte aligned: search it only when the batch has FP32 items
  bool any_f32 = false;
  for (const auto& it : b->items) any_f32 = any_f32 || it.dev.dtype == DT_F32;
  const int32_t widths[] = {32, 16};
  const int nwidths = any_f32 ? 2 : 1;
  float best = 1e30f;
  int32_t bu = b->unroll, bb = b->block, bv = b->vec_bytes;
  int64_t bt = b->tile_bytes;
  salt_status st = SALT_OK;
  for (int wi = 0; wi < nwidths && st == SALT_OK; ++wi) {
    st = salt_batch_set_vec_bytes(b, widths[wi]);
    for (int32_t u : unrolls) {
      if (st != SALT_OK) break;
      for (int32_t blk : blocks) {
        for (int64_t t : tiles) {
          st = salt_batch_set_config(b, u, blk, 0, t);
          if (st != SALT_OK) break;
          st = launch(b, red_out, s);  // warm-up (builds the table and graph)
          if (st != SALT_OK) break;
          cudaEventRecord(e0, s);
          for (int r = 0; r < reps && st == SALT_OK; ++r) st = launch(b, red_out, s);
          cudaEventRecord(e1, s);
          if (st != SALT_OK) break;
          if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(SALT_ERR_CUDA, "cudaEventSynchronize");
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          ms /= (float)reps;
          if (ms < best) {
            best = ms;
            bu = u;
            bb = blk;
            bt = t;
            bv = widths[wi];
          }
        }
        if (st != SALT_OK) break;
      }
      if (st != SALT_OK) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SALT_OK) return st;
  st = salt_batch_set_vec_bytes(b, bv);
  if (st == SALT_OK) st = salt_batch_set_config(b, bu, bb, 0, bt);
  if (best_ms) *best_ms = best;
  return st;
}

}  // extern "C"
