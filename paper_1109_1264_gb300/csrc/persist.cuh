// Persistent serving kernel (salt_serve_* with `persistent` set): the blocks
// stay resident and run the steps the host posts to a ring in mapped host
// memory, so a step costs no launch, no table upload through a copy engine
// and no event.  One launch runs steps first_step, first_step + 1, ... :
//
//   block 0   (the dispatcher, which takes no tiles) waits (bounded) until
//             the step two before is complete (the device tables, tile
//             counters and partials alternate between two sets by step
//             parity), then until the host has posted the step (or asked to
//             stop, or nothing came for idle_ns: the launch ends), copies the
//             step's tables from the ring entry into its set and releases
//             the step (sync[0] = step), usually while the workers still run
//             the step before;
//   workers   (every other block) wait (bounded) for that release, then run
//             the fill phase (when the step has fill items) and the compute
//             phase with the batch kernel's tile loop; between the phases
//             every worker waits (bounded) for the last one; the compute
//             phase's last worker publishes the step's completion to the
//             host (ctl->done).
//
// A worker that has taken its last tile of a step goes on to the next step
// while others finish theirs, so consecutive steps overlap (like steps on
// two streams).  Completion stays in step order: a step's last arrival comes
// after every worker's arrival in the step before.
//
// A wait that runs out sets ctl->status and the launch ends.  The host
// relaunches the kernel when it has posted a step and the previous launch
// has ended.  Every loop below is bounded by a time limit on %globaltimer
// and by a poll count.
#pragma once

#include "batch.cuh"

namespace salt {

constexpr unsigned kPersistTimeout = 1u;  // ctl->status: a bounded wait ran out
constexpr int kStepHead = 256;            // bytes of the StepDesc slot at the start of a ring entry
constexpr int kHdrSlot = 256;             // bytes per BatchHeader slot

// Control block in mapped pinned host memory.
struct PersistCtl {
  unsigned long long posted;     // host: steps posted so far (step s is in ring entry (s - 1) % nring)
  unsigned long long done;       // kernel: steps complete (results visible to the host)
  unsigned stop;                 // host: end the launch once every posted step is done
  unsigned status;               // kernel: kPersistTimeout
  unsigned long long fail_step;  // kernel: the step a wait ran out in
};

// Start of a ring entry: [StepDesc | hdr fill | hdr compute | fill items | compute items].
struct StepDesc {
  unsigned long long used;          // bytes in use (a multiple of 16)
  unsigned long long off_items[2];  // offsets of the fill and compute item tables
};

struct PersistParams {
  PersistCtl* ctl;                    // device address of the control block
  const char* ring;                   // device address of ring entry 0 (mapped host memory)
  unsigned long long entry_bytes;     // stride between ring entries
  double* red;                        // device address of ring entry 0's results (mapped host memory)
  unsigned long long red_stride;      // doubles per ring entry
  unsigned long long nring;
  char* table;                        // two device copies of ring entries (entry_bytes each), by step parity
  unsigned* counters;                 // per parity and phase: tile counter, arrivals, per-item tickets
  unsigned long long counters_stride; // unsigned per (parity, phase)
  double* partials;                   // per parity: partials_stride doubles
  unsigned long long partials_stride;
  unsigned long long* sync;           // [0] step released, [1] epoch of an exit, [2 + ph] step whose phase ph is complete
  unsigned long long first_step;      // this launch's first step (steps complete + 1)
  unsigned long long epoch;           // this launch's number
  unsigned long long idle_ns;         // block 0 ends the launch after this long with nothing posted
  unsigned long long wait_ns;         // bound on every other wait
  unsigned long long max_polls;       // bound on the polls of every wait
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Waits until *w >= v (device memory).  False when the time or poll bound
// ran out first.
__device__ __forceinline__ bool wait_ge(const unsigned long long* w, unsigned long long v, unsigned long long limit_ns,
                                        unsigned long long max_polls) {
  const unsigned long long t0 = global_ns();
  for (unsigned long long polls = 0;; ++polls) {
    if (ld_acquire_gpu(w) >= v) return true;
    if (polls >= max_polls || global_ns() - t0 > limit_ns) return false;
    __nanosleep(128);
  }
}

// Block 0, thread 0: waits for step s to be posted.  0: posted; 1: the host
// asked to stop, or nothing was posted for idle_ns (either way the launch
// ends; the host relaunches when it posts again).
__device__ __forceinline__ int wait_posted(const PersistParams& p, unsigned long long s) {
  const unsigned long long t0 = global_ns();
  for (unsigned long long polls = 0;; ++polls) {
    if (ld_acquire_sys(&p.ctl->posted) >= s) return 0;
    if (*(volatile unsigned*)&p.ctl->stop) return 1;
    if (polls >= p.max_polls || global_ns() - t0 > p.idle_ns) return 1;
    __nanosleep(256);
  }
}

// Every worker, thread 0: waits for block 0 to release step s (0) or to end
// the launch (1); 2 when the bound ran out.
__device__ __forceinline__ int wait_release(const PersistParams& p, unsigned long long s) {
  const unsigned long long t0 = global_ns();
  const unsigned long long limit = p.idle_ns + 2 * p.wait_ns;
  for (unsigned long long polls = 0;; ++polls) {
    if (ld_acquire_gpu(&p.sync[0]) >= s) return 0;
    if (ld_acquire_gpu(&p.sync[1]) == p.epoch) return 1;
    if (polls >= p.max_polls || global_ns() - t0 > limit) return 2;
    __nanosleep(256);
  }
}

// Every writer stores the same status, so plain system-visible stores do.
__device__ __forceinline__ void note_timeout(const PersistParams& p, unsigned long long s) {
  *(volatile unsigned long long*)&p.ctl->fail_step = s;
  __threadfence_system();
  *(volatile unsigned*)&p.ctl->status = kPersistTimeout;
  __threadfence_system();
}

// Block 0: copies ring entry (s - 1) % nring into the device table of step
// s's parity (at most entry_bytes, the table's size), with 16-byte volatile loads of the host's
// data (relaxed, system scope; no read-only path: the entry is rewritten for
// later steps).  The first blockDim x 16 bytes are loaded together with the
// entry's size, in one round trip; the rest, if any, eight loads in flight
// per thread.
__device__ __forceinline__ void copy_entry(const PersistParams& p, unsigned long long s) {
  __shared__ unsigned long long s_used;
  const uint4* from = (const uint4*)(p.ring + ((s - 1) % p.nring) * p.entry_bytes);
  uint4* to = (uint4*)(p.table + (s & 1ull) * p.entry_bytes);
  const long long cap = (long long)(p.entry_bytes / 16), first = cap < blockDim.x ? cap : blockDim.x;
  uint4 r0 = make_uint4(0u, 0u, 0u, 0u);
  if ((long long)threadIdx.x < first)
    asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0.x), "=r"(r0.y), "=r"(r0.z), "=r"(r0.w)
                 : "l"(from + threadIdx.x)
                 : "memory");
  if (threadIdx.x == 0) {
    const unsigned long long want = ((unsigned long long)r0.y << 32) | r0.x;  // StepDesc::used
    s_used = want < p.entry_bytes ? want : p.entry_bytes;
  }
  __syncthreads();
  const long long nv = (long long)(s_used / 16);
  if ((long long)threadIdx.x < first && (long long)threadIdx.x < nv) to[threadIdx.x] = r0;
  for (long long base = first; base < nv; base += 8LL * blockDim.x) {
    uint4 r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const long long i = base + (long long)k * blockDim.x + threadIdx.x;
      if (i < nv) {
        asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[k].x), "=r"(r[k].y), "=r"(r[k].z), "=r"(r[k].w)
                     : "l"(from + i)
                     : "memory");
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const long long i = base + (long long)k * blockDim.x + threadIdx.x;
      if (i < nv) to[i] = r[k];
    }
  }
}

template <int U>
__global__ void __launch_bounds__(256, 4) persist_kernel(const PersistParams p) {
  __shared__ int s_cmd;
  if (blockIdx.x == 0) {
    // ---- the dispatcher (block 0, no tiles): releases the steps in order,
    // each as soon as it is posted and the step two before is complete, or
    // ends the launch
    for (unsigned long long s = p.first_step;; ++s) {
      __syncthreads();  // every thread has read s_cmd of the previous step
      if (threadIdx.x == 0) {
        int cmd = 0;
        // the step two before used this parity's tables, counters and partials
        if (s >= p.first_step + 2 && !wait_ge(&p.sync[3], s - 2, p.wait_ns, p.max_polls)) cmd = 2;
        if (cmd == 0) cmd = wait_posted(p, s);
        s_cmd = cmd;
      }
      __syncthreads();
      if (s_cmd == 0) copy_entry(p, s);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (s_cmd == 0) {
          st_release_gpu(&p.sync[0], s);
        } else {
          if (s_cmd == 2) note_timeout(p, s);
          st_release_gpu(&p.sync[1], p.epoch);
        }
      }
      __syncthreads();
      if (s_cmd != 0) return;
    }
  }
  // ---- the workers (blocks 1 ..): the released steps, in order
  const unsigned workers = gridDim.x - 1u;
  for (unsigned long long s = p.first_step;; ++s) {
    __syncthreads();  // every thread has read s_cmd of the previous step
    if (threadIdx.x == 0) {
      const int r = wait_release(p, s);
      if (r == 2) note_timeout(p, s);
      s_cmd = r;
    }
    __syncthreads();
    if (s_cmd != 0) return;
    // the step: fill phase (if any), then compute phase
    const unsigned long long par = s & 1ull;
    const char* tab = p.table + par * p.entry_bytes;
    const StepDesc* d = (const StepDesc*)tab;
    for (int ph = 0; ph < 2; ++ph) {
      const BatchHeader* hdr = (const BatchHeader*)(tab + kStepHead + kHdrSlot * ph);
      if (ph == 0 && hdr->nitems == 0) continue;  // the same decision in every worker
      unsigned* cnt = p.counters + (par * 2 + (unsigned long long)ph) * p.counters_stride;
      const BatchParams bp{hdr,
                           (const BatchItem*)(tab + d->off_items[ph]),
                           cnt,
                           cnt + 1,
                           cnt + 2,
                           p.partials + par * p.partials_stride,
                           p.red + ((s - 1) % p.nring) * p.red_stride};
      run_tiles<U, false>(bp);
      __syncthreads();
      if (threadIdx.x == 0) {
        // The arrival releases this block's writes (results in mapped host
        // memory included) at GPU scope; the last worker acquires every
        // arrival, and its system-scope release of ctl->done passes them on
        // to the host (causality order is transitive across the scopes).
        const bool last = ticket_add_acq_rel(cnt + 1, 1u) == workers - 1u;
        int r = 0;
        if (last) {
          // every worker has taken its last tile of the phase: counters back to zero
          cnt[0] = 0u;
          cnt[1] = 0u;
          if (ph == 1) st_release_sys(&p.ctl->done, s);
          st_release_gpu(&p.sync[2 + ph], s);
        } else if (ph == 0) {
          // the compute phase reads what the fill phase wrote
          if (!wait_ge(&p.sync[2], s, p.wait_ns, p.max_polls)) {
            note_timeout(p, s);
            r = 2;
          }
        }
        s_cmd = r;
      }
      __syncthreads();
      if (s_cmd != 0) return;
    }
  }
}

}  // namespace salt
