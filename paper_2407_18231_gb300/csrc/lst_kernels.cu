// Stage kernels of the LST chain on sm_103a (arXiv:2407.18231, Sec. 1).
//
// Design: every object-producing stage is a join over small work units (a lower hit, an
// anchor MD, an LS, a T3, a (pLS, MD) item, a pT3) whose candidates are a few contiguous
// index ranges.  A warp takes a unit, or 32 consecutive units, scans their range lengths
// with shuffles, walks the concatenated candidates 32 at a time (each lane finds its unit
// by a shuffle binary search), tests them and counts the passes with ballot + popc.  A
// count pass sizes every unit (keeping pass bits or partner lists where they fit), a
// device-wide scan turns sizes into offsets, and a fill pass writes each unit's slice of
// the output from what the count pass kept, testing again only where nothing was kept.
// Output order is therefore fixed by the inputs (unit order, then candidate order) and
// never by scheduling, no list is truncated, and every object list ends up sorted by its
// first MD -- which makes "all T3s starting on module M" a single contiguous range for
// the pLS joins.  All grids are persistent (a multiple of the SM count) and read their
// sizes from the device-side batch header, so one CUDA graph replays any batch that fits
// the buffers.
#include <cuda_runtime.h>

#include <utility>

#include "../../include/lst.h"
#include "lst_device.cuh"

namespace lst {

constexpr uint32_t FULL = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }


// Programmatic dependent launch: every kernel of the chain is launched so that it may be
// scheduled as soon as its predecessor's blocks have all exited (no explicit trigger: an
// early one let waiting blocks take the slots of the persistent grids and was slower), and
// waits here, before any access to what the predecessor wrote, until that grid's writes
// are visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Number of lanes whose inclusive prefix is <= cand (the lane owning candidate cand).
__device__ __forceinline__ uint32_t owner_lane(uint32_t incl, uint32_t cand) {
  uint32_t o = 0;
#pragma unroll
  for (uint32_t s = 16; s >= 1; s >>= 1) {
    const uint32_t v = __shfl_sync(FULL, incl, o + s - 1);
    if (v <= cand) o += s;
  }
  return o;
}

// Division by a divisor fixed for a launch, for n + d < 2^32: the multiply-high estimate by
// m = ceil(2^32 / d) is floor(n / d) or one more, and one comparison corrects it.
struct FastDiv {
  uint32_t d, m;
  __device__ explicit FastDiv(uint32_t d_) : d(d_), m(d_ > 1 ? (uint32_t)((0x100000000ull + d_ - 1) / d_) : 0u) {}
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    if (d <= 1) return n;
    const uint32_t q = __umulhi(n, m);
    return q * d > n ? q - 1 : q;
  }
};

// Per-warp bump allocator over a scratch arena (one global atomic per 1024+ words).
struct WarpAlloc {
  uint32_t cur = 0, end = 0;  // warp-uniform
  bool full = false;          // a request found the arena exhausted: count needs, stop grabbing
};

// Walks all (outer i, inner j) candidates of one unit 32 at a time; outer(i, begin, count)
// gives the inner index range of outer item i and test(i, j) decides.  Count pass (FILL =
// false): returns the number of passes.  Fill pass: emit(pos, i, j) for each pass, pos =
// base + rank in candidate order.
template <bool FILL, typename OuterFn, typename TestFn, typename EmitFn>
__device__ __forceinline__ uint32_t warp_join(uint32_t n_outer, uint32_t base, OuterFn outer, TestFn test,
                                              EmitFn emit) {
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t count = 0;
  for (uint32_t g0 = 0; g0 < n_outer; g0 += 32) {
    uint32_t b = 0, c = 0;
    if (g0 + lane < n_outer) outer(g0 + lane, b, c);
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t bo = __shfl_sync(FULL, b, o);
      const uint32_t co = __shfl_sync(FULL, c, o);
      const uint32_t io = __shfl_sync(FULL, incl, o);
      const uint32_t j = bo + (cc - (io - co));
      const bool pass = cand < total && test(g0 + o, j);
      const uint32_t bal = __ballot_sync(FULL, pass);
      if (FILL && pass) emit(base + count + __popc(bal & lt), g0 + o, j);
      count += __popc(bal);
    }
  }
  return count;
}

// Does any (outer i, inner j) candidate satisfy test(i, j)?  Same flattened walk as
// warp_join, 32 candidates per step, stopping at the first step with a hit.
template <typename OuterFn, typename TestFn>
__device__ __forceinline__ bool warp_any(uint32_t n_outer, OuterFn outer, TestFn test) {
  const uint32_t lane = lane_id();
  for (uint32_t g0 = 0; g0 < n_outer; g0 += 32) {
    uint32_t b = 0, c = 0;
    if (g0 + lane < n_outer) outer(g0 + lane, b, c);
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t bo = __shfl_sync(FULL, b, o);
      const uint32_t co = __shfl_sync(FULL, c, o);
      const uint32_t io = __shfl_sync(FULL, incl, o);
      const uint32_t j = bo + (cc - (io - co));
      const bool hit = cand < total && test(g0 + o, j);
      if (__any_sync(FULL, hit)) return true;
    }
  }
  return false;
}

// warp_any for groups of S lanes (S a power of two, n_outer <= S): each group answers for
// its own object, so a warp has 32 / S objects' loads in flight.  A group with active ==
// false has no candidates.  Uniform across the warp: every lane must call it.
template <uint32_t S, typename OuterFn, typename TestFn>
__device__ __forceinline__ bool group_any(bool active, uint32_t n_outer, OuterFn outer, TestFn test) {
  static_assert(S >= 2 && S <= 32 && (S & (S - 1)) == 0, "group size");
  const uint32_t r = lane_id() & (S - 1);
  const uint32_t gmask = S == 32 ? FULL : ((1u << (S & 31u)) - 1u) << (lane_id() & ~(S - 1));
  uint32_t b = 0, c = 0;
  if (active && r < n_outer) outer(r, b, c);
  uint32_t incl = c;
#pragma unroll
  for (uint32_t o = 1; o < S; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o, S);
    if (r >= o) incl += t;
  }
  const uint32_t total = __shfl_sync(FULL, incl, S - 1, S);
  bool found = false;
  for (uint32_t t0 = 0; __any_sync(FULL, t0 < total && !found); t0 += S) {
    const uint32_t cand = t0 + r;
    const uint32_t cc = cand < total ? cand : (total ? total - 1 : 0u);
    uint32_t o = 0;
#pragma unroll
    for (uint32_t st = S / 2; st >= 1; st >>= 1) {
      const uint32_t v = __shfl_sync(FULL, incl, o + st - 1, S);
      if (v <= cc) o += st;
    }
    const uint32_t bo = __shfl_sync(FULL, b, o, S);
    const uint32_t co = __shfl_sync(FULL, c, o, S);
    const uint32_t io = __shfl_sync(FULL, incl, o, S);
    const bool hit = !found && cand < total && test(o, bo + (cc - (io - co)));
    if (__ballot_sync(FULL, hit) & gmask) found = true;
  }
  return found;
}

__device__ __forceinline__ uint32_t find_slot(const uint32_t* off, uint32_t n, uint32_t x) {
  // largest e in [0, n) with off[e] <= x (off non-decreasing, off[0] = 0)
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

#define WARP_LOOP(unit, n)                                                                         \
  for (uint32_t unit = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; unit < (n);                   \
       unit += (gridDim.x * blockDim.x) >> 5)
// Dynamic scheduling for joins whose units differ widely in cost: warps take batches of G
// units from a counter in the header (zeroed with every launch) and request the next batch
// before working on the current one, so the atomic's latency overlaps the work.  When the
// units are few (at most 4 batches per warp: one event) a warp's first batch is fixed
// instead (warp w takes [w G, w G + G), the counter hands out the rest), which spares the
// burst of atomics at launch that would dominate so short a kernel.  `continue` moves to
// the next unit.
struct WarpQueue {
  uint32_t* ctr;
  uint32_t g, base, cur, pend;
  __device__ __forceinline__ WarpQueue(uint32_t* c, uint32_t grain, uint32_t n) : ctr(c), g(grain), pend(0) {
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    if (n <= 4u * nw * grain) {
      base = nw * grain;
      cur = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * grain;
    } else {
      base = 0;
      issue();
      cur = collect();
    }
  }
  // lane 0 starts the atomic; its result is only read by collect(), after the batch's work
  __device__ __forceinline__ uint32_t issue() {
    if (lane_id() == 0) pend = atomicAdd(ctr, g);
    return cur;
  }
  __device__ __forceinline__ uint32_t collect() { return base + __shfl_sync(0xFFFFFFFFu, pend, 0); }
};
#define DYN_LOOP(k, ctr, n, grain)                                                                       \
  for (WarpQueue wq_(ctr, grain, n); wq_.cur < (n);)                                                   \
    for (uint32_t e_ = min(wq_.cur + (grain), (uint32_t)(n)), k = wq_.issue(); k < e_ || (wq_.cur = wq_.collect(), false); \
         k++)
#define THREAD_LOOP(i, n) \
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)
// One object per group of S lanes; the loop is uniform across the warp (act: this group has
// an object in this round).
#define GROUP_LOOP(x, act, n, S)                                                                          \
  for (uint32_t x##0_ = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / (S)); x##0_ < (n);          \
       x##0_ += ((gridDim.x * blockDim.x) >> 5) * (32 / (S)))                                             \
    for (uint32_t x = x##0_ + (lane_id() / (S)), act = x < (n), once_ = 1; once_; once_ = 0)
// Lanes per object in the duplicate-removal walks (measured: the T5 cross-stage walk gains
// from several objects per warp, the same-stage walks, with longer lists, do not).
constexpr uint32_t CROSS_T5_GROUP = 16, KILL_T5_GROUP = 32, KILL_PT5_GROUP = 32;

// ------------------------------------------------------------------ scans
// Exclusive scan of n = (*nptr) * mul u32 values into out[0..n], out[n] = total; the total
// goes to hdr->tot[tot] and a total above cap raises that list's overflow bit.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sm, uint32_t& total) {
  const uint32_t lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31) sm[w] = incl;
  __syncthreads();
  if (w == 0) {
    const uint32_t x = lane < nw ? sm[lane] : 0u;
    const uint32_t xi = warp_incl_scan(x);
    sm[lane] = xi - x;
    if (lane == 31) sm[32] = xi;
  }
  __syncthreads();
  const uint32_t r = sm[w] + incl - v;
  total = sm[32];
  __syncthreads();
  return r;
}

// Every scan writes out[0..n) (exclusive), out[n] = total, the header total and its
// overflow bit.  One block scans a whole array when the array's capacity is at most
// SCAN_SMALL_MAX (the lists of a small event): tiles of 16 elements per thread with a
// running carry, no waiting on other blocks.  Measured: 7 us for one tile; at 60 k elements
// (4 tiles) 22 us, slower than the multi-block single pass below, so the bound is one tile.
constexpr uint32_t SCAN_SMALL_MAX = 1u << 14;
constexpr uint32_t SCAN_SMALL_PER_THREAD = 16;
__device__ __forceinline__ void scan_small_body(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ out,
                                                Hdr* H, int tot_idx, uint32_t cap, uint32_t* sm) {
  uint32_t carry = 0;
  for (uint32_t t = 0; t < n; t += blockDim.x * SCAN_SMALL_PER_THREAD) {
    const uint32_t i0 = t + threadIdx.x * SCAN_SMALL_PER_THREAD;
    uint32_t v[SCAN_SMALL_PER_THREAD];
    uint32_t s = 0;
#pragma unroll
    for (uint32_t k = 0; k < SCAN_SMALL_PER_THREAD; k++) {
      v[k] = (i0 + k < n) ? in[i0 + k] : 0u;
      s += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(s, sm, tot) + carry;
#pragma unroll
    for (uint32_t k = 0; k < SCAN_SMALL_PER_THREAD; k++) {
      if (i0 + k < n) out[i0 + k] = ex;
      ex += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0) {
    out[n] = carry;
    if (tot_idx >= 0) {
      H->tot[tot_idx] = carry;
      if (carry > cap) atomicOr(&H->err, 1u << (ERR_OVERFLOW_SHIFT + tot_idx));
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan_small(const uint32_t* __restrict__ in, const uint32_t* nptr,
                                                     uint32_t mul, Hdr* H, uint32_t* __restrict__ out, int tot_idx,
                                                     uint32_t cap) {
  pdl_wait();
  if (H->err) return;
  __shared__ uint32_t sm[33];
  scan_small_body(in, (*nptr) * mul, out, H, tot_idx, cap, sm);
}

constexpr uint32_t SCAN_WAIT_LIMIT = 1u << 20;  // about a second of polls
static_assert(11 + 4 <= N_SCAN_SLOTS, "scan slots: eight single scans, then three and four arrays");

// Larger arrays (capacity above SCAN_SMALL_MAX: one event's or a batch's lists): a single pass with one
// chunk of SCAN_LARGE_CHUNK elements (1024 threads x 8) per block.  A block takes a ticket
// when it starts (its chunk, so chunks are handed out in start order), publishes its chunk's
// total at once, then looks back over the chunks before its own, 32 at a time, adding their
// totals until it meets one that has published its inclusive prefix, and publishes its own
// (decoupled look-back).  A chunk state is [run number | flag | value]: states of earlier
// runs read as not yet written, so the state array is never cleared between runs.  A block
// waits only for blocks that started before it, and every wait is bounded
// (SCAN_WAIT_LIMIT polls, then ERR_WAIT, the wait taken as an inclusive prefix of 0).
constexpr unsigned long long ST_AGG = 1ull << 32, ST_INCL = 2ull << 32, ST_FLAGS = 3ull << 32;
constexpr uint32_t SCAN_LARGE_PER_THREAD = SCAN_LARGE_CHUNK / 1024;
static_assert(SCAN_LARGE_PER_THREAD == 8, "two 16-byte loads and stores per thread");
__device__ __forceinline__ void scan_large_body(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ out,
                                                Hdr* H, int tot_idx, uint32_t cap, uint32_t slot, const BufView& B,
                                                uint32_t* sm) {
  if (threadIdx.x == 0) sm[33] = atomicAdd(&H->scan_ticket[slot], 1u);
  __syncthreads();
  const uint32_t b = sm[33];
  const uint32_t nch = max(1u, (n + SCAN_LARGE_CHUNK - 1) / SCAN_LARGE_CHUNK);  // chunk 0 also when n = 0
  if (b >= nch) return;  // (block-uniform) a block past the last chunk
  if (b >= B.scan_chunks || B.scan_state == nullptr) {  // cannot happen: the states are sized from the capacities
    if (threadIdx.x == 0) atomicOr(&H->err, ERR_WAIT);
    return;
  }
  unsigned long long* st = B.scan_state + (size_t)slot * B.scan_chunks;
  const unsigned long long tag = (unsigned long long)(H->scan_epoch & 0x3FFFFFFFu) << 34;
  const uint32_t lo = b * SCAN_LARGE_CHUNK, hi = min(n, lo + SCAN_LARGE_CHUNK);
  const uint32_t i0 = lo + threadIdx.x * SCAN_LARGE_PER_THREAD;
  const bool vec = i0 + SCAN_LARGE_PER_THREAD <= hi &&
                   ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
  uint32_t v[SCAN_LARGE_PER_THREAD];
  if (vec) {
    const uint4 a = *reinterpret_cast<const uint4*>(in + i0), c = *reinterpret_cast<const uint4*>(in + i0 + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = c.x; v[5] = c.y; v[6] = c.z; v[7] = c.w;
  } else {
#pragma unroll
    for (uint32_t k = 0; k < SCAN_LARGE_PER_THREAD; k++) v[k] = (i0 + k < hi) ? in[i0 + k] : 0u;
  }
  uint32_t s = 0;
#pragma unroll
  for (uint32_t k = 0; k < SCAN_LARGE_PER_THREAD; k++) s += v[k];
  uint32_t tot;
  uint32_t ex = block_excl_scan(s, sm, tot);
  if (threadIdx.x < 32) {
    const uint32_t lane = threadIdx.x;
    uint32_t prefix = 0;
    if (b > 0) {
      if (lane == 0) atomicExch(&st[b], tag | ST_AGG | tot);
      for (int32_t j = (int32_t)b - 1;; j -= 32) {  // warp-uniform
        const int32_t idx = j - (int32_t)lane;
        unsigned long long w = tag | ST_INCL;  // before chunk 0: an inclusive prefix of 0
        if (idx >= 0) {
          uint32_t it = 0;
          for (; it < SCAN_WAIT_LIMIT; it++) {
            w = atomicAdd(&st[idx], 0ull);
            if ((w >> 34) == (tag >> 34) && (w & ST_FLAGS)) break;
          }
          if (it == SCAN_WAIT_LIMIT) {
            atomicOr(&H->err, ERR_WAIT);
            w = tag | ST_INCL;
          }
        }
        const uint32_t im = __ballot_sync(FULL, (w & ST_FLAGS) == ST_INCL);
        const uint32_t upto = im ? (uint32_t)__ffs(im) - 1u : 31u;  // the nearest inclusive prefix ends the walk
        prefix += __reduce_add_sync(FULL, lane <= upto ? (uint32_t)w : 0u);
        if (im) break;
      }
    }
    if (lane == 0) {
      atomicExch(&st[b], tag | ST_INCL | (uint32_t)(prefix + tot));
      sm[34] = prefix;
    }
  }
  __syncthreads();
  const uint32_t carry = sm[34];
  ex += carry;
  if (vec) {
    uint32_t o[SCAN_LARGE_PER_THREAD];
#pragma unroll
    for (uint32_t k = 0; k < SCAN_LARGE_PER_THREAD; k++) {
      o[k] = ex;
      ex += v[k];
    }
    *reinterpret_cast<uint4*>(out + i0) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4*>(out + i0 + 4) = make_uint4(o[4], o[5], o[6], o[7]);
  } else {
#pragma unroll
    for (uint32_t k = 0; k < SCAN_LARGE_PER_THREAD; k++) {
      if (i0 + k < hi) out[i0 + k] = ex;
      ex += v[k];
    }
  }
  if (b == nch - 1 && threadIdx.x == 0) {
    const uint32_t total = carry + tot;
    out[n] = total;
    if (tot_idx >= 0) {
      H->tot[tot_idx] = total;
      if (total > cap) atomicOr(&H->err, 1u << (ERR_OVERFLOW_SHIFT + tot_idx));
    }
  }
}

__global__ void __launch_bounds__(1024) k_scan_large(const uint32_t* __restrict__ in, const uint32_t* nptr,
                                                     uint32_t mul, BufView B, uint32_t* __restrict__ out, int tot_idx,
                                                     uint32_t cap, uint32_t slot) {
  pdl_wait();
  Hdr* H = B.hdr;
  if (H->err) return;
  __shared__ uint32_t sm[35];
  scan_large_body(in, (*nptr) * mul, out, H, tot_idx, cap, slot, B, sm);
}

// Up to four independent scans in one launch (blockIdx.y picks the array).
struct ScanJob {
  const uint32_t* in;
  uint32_t* out;
  const uint32_t* nptr;
  int tot;
  uint32_t cap;
};
struct ScanJobs {
  ScanJob j[4];
};

// The one-block scan of several small arrays (blockIdx.x picks the array).
__global__ void __launch_bounds__(1024) k_scan_small_multi(ScanJobs J, Hdr* H) {
  pdl_wait();
  if (H->err) return;
  __shared__ uint32_t sm[33];
  const ScanJob& q = J.j[blockIdx.x];
  scan_small_body(q.in, *q.nptr, q.out, H, q.tot, q.cap, sm);
}

// The single-pass scan of several large arrays (blockIdx.y picks the array and its slot).
__global__ void __launch_bounds__(1024) k_scan_large_multi(ScanJobs J, BufView B, uint32_t slot0) {
  pdl_wait();
  Hdr* H = B.hdr;
  if (H->err) return;
  __shared__ uint32_t sm[35];
  const ScanJob& q = J.j[blockIdx.y];
  scan_large_body(q.in, *q.nptr, q.out, H, q.tot, q.cap, slot0 + blockIdx.y, B, sm);
}

__global__ void k_zero(uint32_t* p, const uint32_t* nptr, uint32_t mul, uint32_t add) {
  pdl_wait();
  const uint32_t n = (*nptr) * mul + add;
  THREAD_LOOP(i, n) p[i] = 0u;
}

// ------------------------------------------------------------------ hit binning
// Count hits per (event, sensor); validate module ids and coordinates.
__global__ void k_hits_count(GeoView G, BufView B) {
  pdl_wait();
  Hdr* H = B.hdr;
  const uint32_t n = H->n_hits, ne = H->n_ev, two_nm = 2u * G.nm;
  THREAD_LOOP(h, n) {
    const uint32_t e = find_slot(H->hit_off, ne, h);
    const uint32_t det = H->det[h];
    const float x = H->x[h], y = H->y[h], z = H->z[h];
    B.hit_ev[h] = e;
    if (det >= two_nm || !isfinite(x) || !isfinite(y) || !isfinite(z)) {
      atomicOr(&H->err, ERR_BAD_INPUT);
      continue;
    }
    atomicAdd(&B.sen_cnt[e * two_nm + det], 1u);
  }
}

__global__ void k_hits_scatter(GeoView G, BufView B) {
  pdl_wait();
  Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_hits, two_nm = 2u * G.nm;
  THREAD_LOOP(h, n) {
    const uint32_t bkt = B.hit_ev[h] * two_nm + H->det[h];
    const uint32_t pos = B.sen_off[bkt] + atomicSub(&B.sen_cnt[bkt], 1u) - 1u;
    B.hit_tmp[pos] = h;
    B.hit_psi[pos] = pseudo_angle(H->x[h], H->y[h]);
  }
}

// Order inside each sensor bucket: by pseudo-angle (azimuth), ties by input index.
__global__ void k_hits_sort(GeoView G, BufView B) {
  pdl_wait();
  Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_hits, two_nm = 2u * G.nm;
  THREAD_LOOP(p, n) {
    const uint32_t h = B.hit_tmp[p];
    const uint32_t e = B.hit_ev[h];
    const uint32_t bkt = e * two_nm + H->det[h];
    const uint32_t lo = B.sen_off[bkt], hi = B.sen_off[bkt + 1];
    const float x = H->x[h], y = H->y[h], z = H->z[h];
    const float ph = B.hit_psi[p];
    uint32_t rank = 0;
    for (uint32_t q = lo; q < hi; q++) {
      const uint32_t g = B.hit_tmp[q];
      const float pg = B.hit_psi[q];
      rank += (pg < ph) || (pg == ph && g < h);
    }
    B.hit4[lo + rank] = make_float4(x, y, z, sqrtf(x * x + y * y));
    B.hit_idx[lo + rank] = h - H->hit_off[e];
    B.hit_sen[lo + rank] = bkt;
  }
}

// ------------------------------------------------------------------ Mini Doublets
// Candidates of unit (event, module) = lower-sensor hits x upper-sensor hits (Sec. 1).
__device__ __forceinline__ bool md_test(const MethodConst& C, const float4& cst, const float4& lo, const float4& up) {
  const PointTol a{lo, cst}, b{up, cst};
  return pair_rz(C, a, b) && pair_bend(C, a, b, cst.w);
}

__device__ __forceinline__ void md_emit(const BufView& B, uint32_t pos, uint32_t u, uint32_t ih, uint32_t jh,
                                        const float4& hl, const float4& hu, const float4& cst) {
  B.md_unit[pos] = u;
  B.md_pt[2 * (size_t)pos] = hl;
  B.md_up4[pos] = hu;
  B.md_pt[2 * (size_t)pos + 1] = cst;
  B.md_dir4[pos] = md_direction(hl, hu, cst);
  B.md_psi[pos] = pseudo_angle(hl.x, hl.y);
  B.md_lo_idx[pos] = B.hit_idx[ih];
  B.md_up_idx[pos] = B.hit_idx[jh];
}

constexpr uint32_t MD_BIG = 1u << 26;  // candidates of one lower hit above which it is walked alone

// Items are the positions of the sorted hit array: a lower-sensor hit pairs with every
// upper-sensor hit of its unit (event, module) (Sec. 1); an upper-sensor hit has none.  The
// count pass writes each item's passes, and their scan over hit positions orders the MDs
// unit-major and lower-hit-major within a unit (the canonical order).
//
// Count pass: a warp takes 32 items -- slot s owns item s P mod n (P prime, not a divisor of
// n: a permutation), so the lower hits of the busy inner-layer modules spread over all
// warps -- and walks their concatenated candidates 32 at a time.  An item's candidates in a
// chunk are a contiguous lane range, so its passes are popc(ballot & range), and the pass
// bits of its first 32 candidates are kept for the fill pass.
__global__ void __launch_bounds__(512) k_md_count(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_hits;
  const uint32_t ng = (n + 31) >> 5;
  const uint32_t lane = lane_id();
  DYN_LOOP(grp, &B.hdr->work[W_MD], ng, 2) {
    const uint32_t p = grp * 32 + lane;
    const bool valid = p < n;
    uint32_t up_b = 0, c = 0, mod = 0;
    if (valid) {
      const uint32_t sen = B.hit_sen[p];
      if (!(sen & 1u)) {
        up_b = B.sen_off[sen + 1];
        c = B.sen_off[sen + 2] - up_b;
        mod = (sen >> 1) % G.nm;
      }
    }
    if (__any_sync(FULL, c >= MD_BIG)) {  // one item at a time: the chunk sums stay in range
      for (uint32_t k = 0; k < 32; k++) {
        const uint32_t ck = __shfl_sync(FULL, c, k);
        const uint32_t pk = __shfl_sync(FULL, p, k), ubk = __shfl_sync(FULL, up_b, k);
        const uint32_t modk = __shfl_sync(FULL, mod, k);
        if (ck == 0) continue;
        const float4 cst = G.modc[modk];
        const float4 hl = B.hit4[pk];
        uint32_t run = 0;
        for (uint32_t t0 = 0; t0 < ck; t0 += 32) {
          const uint32_t j = t0 + lane;
          const float4 hu = B.hit4[ubk + (j < ck ? j : 0u)];
          const bool pass = j < ck && md_test(C, cst, hl, hu);
          const uint32_t bal = __ballot_sync(FULL, pass);
          if (t0 == 0 && lane == 0) B.md_hmask[pk] = bal;
          run += __popc(bal);
        }
        if (lane == 0) B.md_hcnt[pk] = run;
      }
      if (valid && c == 0) B.md_hcnt[p] = 0u;
      continue;
    }
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t start = incl - c;  // this lane's item: candidates [start, incl)
    uint32_t run = 0;                 // passes of this lane's item so far
    uint32_t bits = 0;                // pass bits of its first 32 candidates
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t so = __shfl_sync(FULL, start, o);
      const uint32_t po = __shfl_sync(FULL, p, o);
      const uint32_t ubo = __shfl_sync(FULL, up_b, o);
      const uint32_t mo = __shfl_sync(FULL, mod, o);
      const float4 cst = G.modc[mo];
      const float4 hl = B.hit4[po], hu = B.hit4[ubo + (cc - so)];
      const bool pass = cand < total && md_test(C, cst, hl, hu);
      const uint32_t bal = __ballot_sync(FULL, pass);
      // this lane's item's lanes in the chunk: [lo, hi), its candidates t0 + lo - start on
      const uint32_t lo = start > t0 ? min(start - t0, 32u) : 0u;
      const uint32_t hi = incl > t0 ? min(incl - t0, 32u) : 0u;
      if (hi > lo) {
        const uint32_t mine = (bal & (hi == 32u ? FULL : (1u << hi) - 1u)) >> lo;
        run += __popc(mine);
        const uint32_t first = t0 + lo - start;
        if (first < 32u) bits |= mine << first;
      }
    }
    if (valid) {
      B.md_hcnt[p] = run;
      if (c) B.md_hmask[p] = bits;
    }
  }
}

// Fill pass in the natural item order, so that a warp's MDs are consecutive and its stores
// coalesce: a warp takes 32 consecutive items and walks their concatenated passes 32 at a
// time; a pass is the (k+1)-th set bit of its item's stored bits.  An item with more than 32
// candidates (stored bits incomplete) re-tests its candidates instead.  Also writes the
// per-unit MD offsets (the item offset of the unit's first hit).
__global__ void __launch_bounds__(512) k_md_fill(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_hits;
  {
    const uint32_t nu = H->n_ev * G.nm;
    THREAD_LOOP(u, nu + 1) B.md_off[u] = B.md_hoff[B.sen_off[2 * u]];
  }
  const uint32_t ng = (n + 31) >> 5;
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  WARP_LOOP(grp, ng) {
    const uint32_t p = grp * 32 + lane;
    uint32_t base = 0, np = 0, up_b = 0, c = 0, u = 0, mod = 0, bits = 0;
    if (p < n) {
      base = B.md_hoff[p];
      np = B.md_hoff[p + 1] - base;
      if (np) {  // a lower hit
        const uint32_t sen = B.hit_sen[p];
        up_b = B.sen_off[sen + 1];
        c = B.sen_off[sen + 2] - up_b;
        u = sen >> 1;
        mod = u % G.nm;
        bits = B.md_hmask[p];
      }
    }
    const bool small = c <= 32u;
    const uint32_t ns = small ? np : 0u;
    const uint32_t incl = warp_incl_scan(ns);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t k = cc - (__shfl_sync(FULL, incl, o) - __shfl_sync(FULL, ns, o));
      uint32_t m = __shfl_sync(FULL, bits, o);
      const uint32_t po = grp * 32 + o;
      const uint32_t ubo = __shfl_sync(FULL, up_b, o);
      const uint32_t uo = __shfl_sync(FULL, u, o);
      const uint32_t mo = __shfl_sync(FULL, mod, o);
      const uint32_t bo = __shfl_sync(FULL, base, o);
      if (cand < total) {
        for (uint32_t i = 0; i < k; i++) m &= m - 1u;
        const uint32_t jh = ubo + (uint32_t)(__ffs(m) - 1);
        const float4 cst = G.modc[mo];
        md_emit(B, bo + k, uo, po, jh, B.hit4[po], B.hit4[jh], cst);
      }
    }
    // items with more than 32 candidates: re-test, one item at a time
    for (uint32_t big = __ballot_sync(FULL, np && !small); big; big &= big - 1u) {
      const uint32_t k = __ffs(big) - 1;
      const uint32_t ck = __shfl_sync(FULL, c, k), ubk = __shfl_sync(FULL, up_b, k);
      const uint32_t uk = __shfl_sync(FULL, u, k), modk = __shfl_sync(FULL, mod, k);
      const uint32_t bk = __shfl_sync(FULL, base, k);
      const uint32_t pk = grp * 32 + k;
      const float4 cst = G.modc[modk];
      const float4 hl = B.hit4[pk];
      uint32_t run = 0;
      for (uint32_t t0 = 0; t0 < ck; t0 += 32) {
        const uint32_t j = t0 + lane;
        const uint32_t jh = ubk + (j < ck ? j : 0u);
        const float4 hu = B.hit4[jh];
        const bool pass = j < ck && md_test(C, cst, hl, hu);
        const uint32_t bal = __ballot_sync(FULL, pass);
        if (pass) md_emit(B, bk + run + __popc(bal & lt), uk, pk, jh, hl, hu, cst);
        run += __popc(bal);
      }
    }
  }
}

__device__ __forceinline__ PointTol md_point(const BufView& B, uint32_t m) {
  return PointTol{B.md_pt[2 * (size_t)m], B.md_pt[2 * (size_t)m + 1]};
}
__device__ __forceinline__ PointTol md_upper(const BufView& B, uint32_t m) {
  return PointTol{B.md_up4[m], B.md_pt[2 * (size_t)m + 1]};
}

// ------------------------------------------------------------------ Line Segments
// The LS selection of ls_select for anchor pa and MD j, loading the rest of MD j
// only when the cheap tests pass.
// Split in two so that a warp can queue the candidates passing the cheap head and run the
// tail only on full warps: ls_test = ls_head && ls_tail.
__device__ __forceinline__ bool ls_head_pt(const MethodConst& C, const PointTol& pa, const PointTol& pb) {
  return pair_rz(C, pa, pb) && pair_bend(C, pa, pb, pb.t.w);
}

__device__ __forceinline__ bool ls_head(const MethodConst& C, const BufView& B, const PointTol& pa, uint32_t j) {
  return ls_head_pt(C, pa, md_point(B, j));
}

// The rest of ls_select after the head: the barrel exit when the pair goes from a barrel
// module to a disk (`exit`), then both MD directions against the chord, from the
// directions stored per MD (da: the anchor's).
__device__ __forceinline__ bool ls_tail_k(const MethodConst& C, const GeoView& G, const BufView& B, const PointTol& pa,
                                          const float4& da, float rnext, bool exit, uint32_t j) {
  const PointTol pb = md_point(B, j);
  if (exit && !exit_ok(pa, pb, rnext, G.zb_half)) return false;
  const float4 db = B.md_dir4[j];
  const float cx = pb.p.x - pa.p.x;
  const float cy = pb.p.y - pa.p.y;
  const float clen = sqrtf(cx * cx + cy * cy);
  return md_dir_pre(C, da, cx, cy, clen) && md_dir_pre(C, db, cx, cy, clen);
}

__device__ __forceinline__ bool ls_tail(const MethodConst& C, const GeoView& G, const BufView& B, const PointTol& pa,
                                        const float4& da, float rnext, bool a_barrel, uint32_t ubase, uint32_t j) {
  return ls_tail_k(C, G, B, pa, da, rnext, a_barrel && G.subdet[B.md_unit[j] - ubase] == 1, j);
}

__device__ __forceinline__ bool ls_test(const MethodConst& C, const GeoView& G, const BufView& B, const PointTol& pa,
                                        const float4& da, float rnext, bool a_barrel, uint32_t ubase, uint32_t j) {
  return ls_head(C, B, pa, j) && ls_tail(C, G, B, pa, da, rnext, a_barrel, ubase, j);
}

// Per-MD LS join (candidates = MDs of every module in the connection map of A): the count
// pass uses it for modules whose flattened neighbour list does not fit the shared-memory
// list, the fill pass for anchors without a stored partner list.
template <bool FILL>
__device__ __forceinline__ void ls_md_join(const MethodConst& C, const GeoView& G, const BufView& B, uint32_t a,
                                           uint32_t ev, uint32_t A) {
  const PointTol pa = md_point(B, a);
  const float4 da = B.md_dir4[a];
  const float rnext = G.rnext[A];
  const bool a_barrel = G.subdet[A] == 0;
  const uint32_t nb0 = G.conn_off[A], nb = G.conn_off[A + 1] - nb0;
  const uint32_t base = FILL ? B.ls_off[a] : 0u;
  const uint32_t ubase = ev * G.nm;
  const uint32_t cnt = warp_join<FILL>(
      nb, base,
      [&](uint32_t i, uint32_t& b, uint32_t& c) {
        const uint32_t u = ubase + G.conn[nb0 + i];
        b = B.md_off[u];
        c = B.md_off[u + 1] - b;
      },
      [&](uint32_t, uint32_t j) { return ls_test(C, G, B, pa, da, rnext, a_barrel, ubase, j); },
      [&](uint32_t pos, uint32_t, uint32_t j) {
        B.ls_in[pos] = a;
        B.ls_out[pos] = j;
      });
  // no partner list is stored for an anchor joined here: the fill pass joins it again
  if (!FILL && lane_id() == 0) {
    B.ls_cnt[a] = cnt;
    B.mask_off[a] = NONE;
  }
}

// LS fill pass, flat over anchor MDs in their order, so that a warp's LSs are consecutive
// and its stores coalesce: a warp takes 32 consecutive anchors and walks their
// concatenated partner lists (stored by the count pass) 32 LSs at a time.  An anchor whose
// list the count pass could not store (arena full, or a neighbour list beyond the shared
// memory) is joined again on its own.
__global__ void __launch_bounds__(512) k_ls_fill(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_MD];
  const uint32_t lane = lane_id();
  WARP_LOOP(grp, (n + 31) >> 5) {
    const uint32_t a = grp * 32 + lane;
    uint32_t base = 0, cnt = 0, mb = NONE;
    if (a < n) {
      base = B.ls_off[a];
      cnt = B.ls_off[a + 1] - base;
      if (cnt) mb = B.mask_off[a];
    }
    const uint32_t ns = mb != NONE ? cnt : 0u;
    const uint32_t incl = warp_incl_scan(ns);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t k = cc - (__shfl_sync(FULL, incl, o) - __shfl_sync(FULL, ns, o));
      const uint32_t bo = __shfl_sync(FULL, base, o);
      const uint32_t mo = __shfl_sync(FULL, mb, o);
      if (cand < total) {
        B.ls_in[bo + k] = grp * 32 + o;
        B.ls_out[bo + k] = B.mask[mo + 1 + k];
      }
    }
    for (uint32_t re = __ballot_sync(FULL, cnt && mb == NONE); re; re &= re - 1u) {
      const uint32_t ak = grp * 32 + __ffs(re) - 1;
      const uint32_t u = B.md_unit[ak];
      const uint32_t ev = u / G.nm;
      ls_md_join<true>(C, G, B, ak, ev, u - ev * G.nm);
    }
  }
}

// Flattened neighbour MDs per warp in shared memory: the launch's list_cap, at most
// LS_LIST_MAX = 64 x 32 (two pass-bit words per lane).  Every list of a PU200-like event fits
// in 512; high-occupancy events reach about 1100, 1500 with tilted modules.
static_assert(LS_LIST_MAX <= 64 * 32, "two pass-bit words per lane");
constexpr uint32_t LS_ANCHORS = 8;     // MDs of a module tested per walk over its list
constexpr uint32_t LS_SPLIT = 4;       // units per module in batches of fewer than 8 events
constexpr uint32_t LS_SPLIT_MIN_HITS = 16384;  // ... that hold at least this many hits
constexpr uint32_t LS_DENSE_HITS = 100000;      // hits per event above which units go one at a time
constexpr uint32_t LS_RING = 64;       // ring of queued (list position, anchor) entries (> 31 + 32)
// per warp after the list: the ring, one pass bit per list position for each anchor, and
// the anchors (lower hit and direction terms: two float4 each; the tolerances are the
// module's, the same for every anchor); list_cap is a multiple of 4, so the anchors' float4s
// stay 16-byte aligned
__host__ __device__ constexpr uint32_t ls_warp_words(uint32_t list_cap) {
  return list_cap + LS_RING + LS_ANCHORS * ((list_cap + 31) / 32) + LS_ANCHORS * 8;
}

// LS count pass.  Unit = (event, module A).  The warp writes the indices of all MDs on the
// modules connected to A into a shared-memory list once (module order, then MD order), then
// walks the list for the MDs a of A: no per-MD neighbour lookups, no per-chunk search.  It
// stores each anchor's partner list (for k_ls_fill to copy) and its count.
__global__ void __launch_bounds__(512) k_ls_count(MethodConst C, GeoView G, BufView B, uint32_t list_cap) {
  pdl_wait();
  extern __shared__ uint32_t ls_smem[];
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t nu = H->n_ev * G.nm;
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* list = ls_smem + (threadIdx.x >> 5) * ls_warp_words(list_cap);
  uint32_t* queue = list + list_cap;
  uint32_t* pbits = queue + LS_RING;
  const uint32_t pw = (list_cap + 31) >> 5;  // pass-bit words per anchor
  float4* anc = reinterpret_cast<float4*>(pbits + LS_ANCHORS * pw);
  WarpAlloc wa;
  // arena pieces a warp takes at least: small enough that every warp of the grid can hold
  // one twice over (a single event's lists need far fewer words than 1024 per warp)
  const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t grab_min = max(32u, min(1024u, B.cap_mask / (2u * n_warps)));
  unsigned long long n_cand = 0;  // count pass: candidate pairs this warp tested
  const uint32_t n_ev = H->n_ev;
  // A small but busy batch has few modules per warp, and its latency is that of the busiest
  // module: there each module's anchor groups are split over LS_SPLIT units (group g in part
  // g mod LS_SPLIT), each walking the module's list for its own groups only.  (A sparse
  // batch would only multiply the work-counter atomics of its mostly empty modules.)
  const uint32_t nsplit = (n_ev < 8 && H->n_hits >= LS_SPLIT_MIN_HITS) ? LS_SPLIT : 1u;
  // events denser than LS_DENSE_HITS hits: units one at a time (their costs differ more)
  const bool dense = H->n_hits >= (uint64_t)LS_DENSE_HITS * n_ev;
  const uint32_t step = nsplit * LS_ANCHORS;
  const FastDiv by_ev(n_ev);
  auto unit = [&](const uint32_t ev, const uint32_t A, const uint32_t part) {
    const uint32_t ubase = ev * G.nm;
    const uint32_t a0 = B.md_off[ubase + A], a1 = B.md_off[ubase + A + 1];
    if (a0 + part * LS_ANCHORS >= a1) return;  // no anchor group in this part
    const uint32_t nb0 = G.conn_off[A], nb = G.conn_off[A + 1] - nb0;
    const float rnext = G.rnext[A];
    const bool a_barrel = G.subdet[A] == 0;
    const float4 t_a = G.modc[A];  // every MD of A carries its module's tolerances
    for (uint32_t ag = a0 + part * LS_ANCHORS; ag < a1; ag += step) {
      const uint32_t na = min(LS_ANCHORS, a1 - ag);
      // The group's anchors span [psi_lo, psi_hi] in pseudo-angle (a module's MDs are in
      // azimuth order), and a candidate on module B can pass the bending cut with one of them
      // only within the edge's half-width (|d psi| <= |d phi|): the list takes, from each
      // connected module, the MDs inside that window (one or, across psi = 0, two runs of its
      // sorted MDs), in module and MD order.
      const float psi_lo = B.md_psi[ag], psi_hi = B.md_psi[ag + na - 1];
      // flattened neighbour list; disk modules have the highest ids, so the disk entries are
      // normally a suffix [t_disk, len) of the list (checked: otherwise each candidate's
      // module is looked up)
      uint32_t len = 0, t_disk = NONE;
      bool suffix = true;
      for (uint32_t g0 = 0; g0 < nb; g0 += 32) {
        uint32_t s1 = 0, e1 = 0, s2 = 0, e2 = 0, c = 0;
        bool disk = false;
        if (g0 + lane < nb) {
          const uint32_t Bm = G.conn[nb0 + g0 + lane];
          const uint32_t uu = ubase + Bm;
          const uint32_t b = B.md_off[uu], end = B.md_off[uu + 1];
          disk = G.subdet[Bm] == 1;
          const float w = G.conn_dpsi[nb0 + g0 + lane];
          const float lo = psi_lo - w, hi = psi_hi + w;
          if (hi - lo >= 4.0f) {  // the whole circle
            s1 = b; e1 = end; s2 = e2 = end;
          } else {
            // window [lo, hi], or [lo + 4, 4) and [0, hi] below 0, or [lo, 4) and [0, hi - 4]
            // above 4: count the sorted MDs below each edge
            const float cut_lo = lo < 0.0f ? lo + 4.0f : lo;
            const float cut_hi = hi >= 4.0f ? hi - 4.0f : hi;
            uint32_t n_lo = 0, n_hi = 0;  // MDs with psi < cut_lo, with psi <= cut_hi
            for (uint32_t i = b; i < end; i++) {
              const float p = B.md_psi[i];
              n_lo += p < cut_lo;
              n_hi += p <= cut_hi;
            }
            if (lo < 0.0f || hi >= 4.0f) {  // two runs: [b, b + n_hi) and [b + n_lo, end)
              s1 = b; e1 = b + n_hi;
              s2 = max(b + n_lo, e1); e2 = end;
            } else {
              s1 = b + n_lo; e1 = max(b + n_hi, s1); s2 = e2 = end;
            }
          }
          c = (e1 - s1) + (e2 - s2);
        }
        const uint32_t incl = warp_incl_scan(c);
        const uint32_t o = len + incl - c;
        uint32_t wpos = o;
        for (uint32_t k = s1; k < e1; k++, wpos++)
          if (wpos < list_cap) list[wpos] = k;
        for (uint32_t k = s2; k < e2; k++, wpos++)
          if (wpos < list_cap) list[wpos] = k;
        const uint32_t dm = __ballot_sync(FULL, disk && c > 0), bm = __ballot_sync(FULL, !disk && c > 0);
        if (t_disk != NONE) {
          if (bm) suffix = false;
        } else if (dm) {
          const uint32_t fd = __ffs(dm) - 1;
          if (fd < 31 && (bm >> (fd + 1))) suffix = false;
          t_disk = __shfl_sync(FULL, o, fd);
        }
        len += __shfl_sync(FULL, incl, 31);
      }
      if (t_disk == NONE) t_disk = len;
      __syncwarp();
      n_cand += (unsigned long long)len * na;
      if (len == 0) {  // no neighbour MD in the window: no LS
        if (lane < na) {
          B.ls_cnt[ag + lane] = 0;
          B.mask_off[ag + lane] = NONE;
        }
        continue;
      }
      if (len > list_cap) {  // recorded, so that the host can give later runs a longer list
        if (lane == 0) atomicMax(&B.hdr->ls_maxlen, len);
        for (uint32_t a = ag; a < ag + na; a++) ls_md_join<false>(C, G, B, a, ev, A);
        continue;
      }
      // Up to LS_ANCHORS MDs of A per walk over the list: their points are staged in shared
      // memory (read as broadcasts) and each candidate loaded is tested against all of
      // them, each anchor with its own pass bits; the head's survivors are queued as
      // list position | anchor << 11 and the tail runs on 32 of them at a time.
      const uint32_t nwords = (len + 31) >> 5;
      // `need` words of the scratch arena from this warp's piece (warp-uniform; NONE when the
      // arena is exhausted: the anchors are then joined again by the fill pass)
      auto alloc = [&](uint32_t need) {
        uint32_t mb = NONE;
        if (lane == 0) {
          if (wa.end - wa.cur < need) {
            if (wa.full) {
              // the arena is exhausted: record only what this list needs ([2]), so the
              // host sizes the next arena from real demand, not from repeated requests
              atomicAdd(&B.hdr->mask_used[2], need);
            } else {
              const uint32_t grab = need > grab_min ? need : grab_min;
              const uint32_t b0 = atomicAdd(&B.hdr->mask_used[1], grab);
              if (b0 < B.cap_mask && grab <= B.cap_mask - b0) {
                wa.cur = b0;
                wa.end = b0 + grab;
              } else {
                wa.cur = wa.end = 0;
                wa.full = true;
                atomicAdd(&B.hdr->mask_used[2], need);
              }
            }
          }
          if (wa.end - wa.cur >= need) {
            mb = wa.cur;
            wa.cur += need;
          }
        }
        wa.cur = __shfl_sync(FULL, wa.cur, 0);
        wa.end = __shfl_sync(FULL, wa.end, 0);
        wa.full = __shfl_sync(FULL, (uint32_t)wa.full, 0) != 0;
        return __shfl_sync(FULL, mb, 0);
      };
      // One anchor's partner list: [count, list entries of its pass bits in list order].
      auto record = [&](uint32_t a, const uint32_t* bits) {
        const uint32_t word = lane < nwords ? bits[lane] : 0u;
        const uint32_t wcnt = __popc(word);
        const uint32_t wincl = warp_incl_scan(wcnt);
        uint32_t count = __shfl_sync(FULL, wincl, 31);
        const uint32_t n_lo = count;
        uint32_t word2 = 0, wcnt2 = 0, wincl2 = 0;
        if (nwords > 32) {  // warp-uniform
          word2 = lane + 32 < nwords ? bits[lane + 32] : 0u;
          wcnt2 = __popc(word2);
          wincl2 = warp_incl_scan(wcnt2);
          count += __shfl_sync(FULL, wincl2, 31);
        }
        uint32_t mbase = NONE;
        if (count > 0) {
          mbase = alloc(1 + count);
          if (mbase != NONE) {
            if (lane == 0) B.mask[mbase] = count;
            uint32_t pos = mbase + 1 + wincl - wcnt;
            for (uint32_t w = word; w; w &= w - 1u) B.mask[pos++] = list[(lane << 5) + __ffs(w) - 1];
            pos = mbase + 1 + n_lo + wincl2 - wcnt2;
            for (uint32_t w = word2; w; w &= w - 1u) B.mask[pos++] = list[((lane + 32) << 5) + __ffs(w) - 1];
          }
        }
        if (lane == 0) {
          B.mask_off[a] = mbase;
          B.ls_cnt[a] = count;
        }
      };
      // All na anchors' lists at once when their pass-bit words fit the warp (lane = anchor k
      // x nwords + word w): one scan and one arena request for the group, the lists laid out
      // one after another in anchor order, each as record() lays it out.
      auto record_group = [&]() {
        const uint32_t k = lane / nwords, w = lane - k * nwords;
        const uint32_t first = k * nwords;  // the lane holding anchor k's first word
        const uint32_t word = k < na ? pbits[k * pw + w] : 0u;
        const uint32_t c = __popc(word);
        const uint32_t incl = warp_incl_scan(c);
        const uint32_t excl = incl - c;
        const uint32_t fl = k < na ? first : 0u, ll = k < na ? first + nwords - 1 : 0u;  // <= 31
        const uint32_t first_excl = __shfl_sync(FULL, excl, fl);
        const uint32_t last_incl = __shfl_sync(FULL, incl, ll);
        const uint32_t count = k < na ? last_incl - first_excl : 0u;
        // anchors with partners, marked at their first lane: each takes one count word
        const uint32_t heads = __ballot_sync(FULL, k < na && w == 0 && count > 0);
        const uint32_t before = __popc(heads & ((1u << fl) - 1u));  // heads of anchors < k
        const uint32_t total = __shfl_sync(FULL, incl, 31) + __popc(heads);
        const uint32_t mbase = total ? alloc(total) : NONE;
        if (mbase != NONE && count > 0) {
          const uint32_t hk = mbase + first_excl + before;  // anchor k's count word
          if (w == 0) B.mask[hk] = count;
          uint32_t pos = hk + 1 + (excl - first_excl);
          for (uint32_t b = word; b; b &= b - 1u) B.mask[pos++] = list[(w << 5) + __ffs(b) - 1];
        }
        if (k < na && w == 0) {
          B.mask_off[ag + k] = count > 0 ? (mbase != NONE ? mbase + first_excl + before : NONE) : NONE;
          B.ls_cnt[ag + k] = count;
        }
      };
      if (lane < na) {
        anc[2 * lane] = B.md_pt[2 * (size_t)(ag + lane)];
        anc[2 * lane + 1] = B.md_dir4[ag + lane];
      }
      for (uint32_t w = lane; w < nwords; w += 32)  // only the words the list covers are used
        for (uint32_t k = 0; k < na; k++) pbits[k * pw + w] = 0;
      uint32_t qh = 0, qt = 0;  // ring head and tail (free-running)
      auto tail = [&](uint32_t e) {
        const uint32_t k = e >> 11, q = e & 2047u;
        const uint32_t j = list[q];
        const bool exit = a_barrel && (suffix ? q >= t_disk : G.subdet[B.md_unit[j] - ubase] == 1);
        const PointTol pa{anc[2 * k], t_a};
        if (ls_tail_k(C, G, B, pa, anc[2 * k + 1], rnext, exit, j))
          atomicOr(&pbits[k * pw + (q >> 5)], 1u << (q & 31));
      };
      __syncwarp();
      for (uint32_t t0 = 0; t0 < len; t0 += 32) {
        const uint32_t t = t0 + lane;
        const uint32_t j = t < len ? list[t] : a0;  // a0: any valid MD for idle lanes
        const PointTol pb{__ldg(&B.md_pt[2 * (size_t)j]), __ldg(&B.md_pt[2 * (size_t)j + 1])};
        for (uint32_t k = 0; k < na; k++) {
          const PointTol pa{anc[2 * k], t_a};
          const bool h = t < len && ls_head_pt(C, pa, pb);
          const uint32_t hb = __ballot_sync(FULL, h);
          if (h) queue[(qt + __popc(hb & lt)) & (LS_RING - 1)] = t | (k << 11);
          qt += __popc(hb);
          if (qt - qh >= 32) {
            __syncwarp();
            tail(queue[(qh + lane) & (LS_RING - 1)]);
            qh += 32;
          }
        }
      }
      __syncwarp();
      if (lane < qt - qh) tail(queue[(qh + lane) & (LS_RING - 1)]);
      __syncwarp();
      if (na * nwords <= 32) {
        record_group();
      } else {
        for (uint32_t k = 0; k < na; k++) record(ag + k, pbits + k * pw);
      }
      __syncwarp();  // the list, anchors, pbits and the queue are reused by the next group
    }
  };
  // module-major order (unit k = part k % nsplit of module k' / n_ev of event k' % n_ev, k' =
  // k / nsplit) taken dynamically: module ids start with the innermost, busiest layers, so
  // expensive units go first; the parts of a module go to different warps (grain 1), and so
  // do the units of dense events, whose busiest modules cost many times the rest
  DYN_LOOP(k, &B.hdr->work[W_LS], nu * nsplit, (nsplit > 1 || dense) ? 1u : 2u) {
    const uint32_t k1 = nsplit > 1 ? k / LS_SPLIT : k;
    const uint32_t A = by_ev.div(k1);
    unit(k1 - A * n_ev, A, k - k1 * nsplit);
  }
  if (lane == 0 && n_cand) atomicAdd(&B.hdr->ls_cand, n_cand);
}

// ------------------------------------------------------------------ T3
// Item = LS l (a -> b), one thread each; candidates = the LSs leaving b (a handful, so a
// thread per LS loads a's and b's records once for all of them).  T3s come out ordered by
// (LS l, LS l2), i.e. by (a, b, c).  The count pass keeps each LS's count and the pass bits
// of its first 32 candidates.
__global__ void __launch_bounds__(512) k_t3_count(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_LS];
  THREAD_LOOP(l, n) {
    const uint32_t a = B.ls_in[l], b = B.ls_out[l];
    const uint32_t c0 = B.ls_off[b], c1 = B.ls_off[b + 1];
    uint32_t cnt = 0, bits = 0;
    if (c0 != c1) {
      const PointTol pa = md_point(B, a), pb = md_point(B, b), pbu = md_upper(B, b);
      for (uint32_t l2 = c0; l2 < c1; l2++) {
        if (t3_select(C, pa, pb, pbu, md_point(B, B.ls_out[l2]))) {
          cnt++;
          if (l2 - c0 < 32) bits |= 1u << (l2 - c0);
        }
      }
    }
    B.t3_lcnt[l] = cnt;
    B.t3_mask[l] = bits;
  }
}

// Fill pass, one thread per LS: with at most 32 candidates the count pass's pass bits say
// which candidates pass (no test), otherwise they are tested again.  Also writes the T3s
// starting at each MD a (those of the LSs leaving a): t3_off[a] = t3_loff[ls_off[a]].
__global__ void __launch_bounds__(512) k_t3_fill(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  THREAD_LOOP(a, H->tot[T_MD] + 1) B.t3_off[a] = B.t3_loff[B.ls_off[a]];
  const uint32_t n = H->tot[T_LS];
  THREAD_LOOP(l, n) {
    uint32_t k = B.t3_loff[l];
    if (B.t3_loff[l + 1] == k) continue;
    const uint32_t a = B.ls_in[l], b = B.ls_out[l];
    const uint32_t c0 = B.ls_off[b], c1 = B.ls_off[b + 1];
    auto emit = [&](uint32_t c) {
      B.t3_a[k] = a;
      B.t3_b[k] = b;
      B.t3_c[k] = c;
      B.t3_md4[k] = make_uint4(a, b, c, 0u);
      k++;
    };
    if (c1 - c0 <= 32) {
      for (uint32_t bits = B.t3_mask[l]; bits; bits &= bits - 1u) emit(B.ls_out[c0 + __ffs(bits) - 1]);
      continue;
    }
    const PointTol pa = md_point(B, a), pb = md_point(B, b), pbu = md_upper(B, b);
    for (uint32_t l2 = c0; l2 < c1; l2++) {
      const uint32_t c = B.ls_out[l2];
      if (t3_select(C, pa, pb, pbu, md_point(B, c))) emit(c);
    }
  }
}

// ------------------------------------------------------------------ T5
// Item = T3 t (a, b, c); candidates = the T3s starting at c.  T5s come out ordered by (T3 t,
// T3 t2), i.e. by (a, b, c, d, e), and t5_toff[t] gives the T5s built on t.  Both passes
// take 32 consecutive T3s per warp and walk their concatenated candidates (count) or
// passes (fill) 32 at a time, so the lanes stay busy whatever the candidate counts.
// The fill pass is a template over the selection (the curvature cuts, or the learned
// selection in their place: select decides and measures, measure only measures); the count
// pass with the learned selection is a kernel of its own, k_t5_count_mlp.
struct T5Cuts {
  __device__ __forceinline__ bool select(const MethodConst& C, const PointTol& A, const PointTol& B,
                                         const PointTol& Cc, const PointTol& D, const PointTol& E, float& score,
                                         float& kfull) const {
    return t5_select(C, A, B, Cc, D, E, score, kfull);
  }
  __device__ __forceinline__ void measure(const MethodConst& C, const PointTol& A, const PointTol& B,
                                          const PointTol& Cc, const PointTol& D, const PointTol& E, float& score,
                                          float& kfull) const {
    t5_select(C, A, B, Cc, D, E, score, kfull);
  }
};
struct T5Net {
  const float* Ws;  // staged weights (t5_mlp_stage)
  __device__ __forceinline__ bool select(const MethodConst& C, const PointTol& A, const PointTol& B,
                                         const PointTol& Cc, const PointTol& D, const PointTol& E, float& score,
                                         float& kfull) const {
    return t5_select_mlp(C, Ws, A, B, Cc, D, E, score, kfull);
  }
  __device__ __forceinline__ void measure(const MethodConst& C, const PointTol& A, const PointTol& B,
                                          const PointTol& Cc, const PointTol& D, const PointTol& E, float& score,
                                          float& kfull) const {
    t5_measure(A, B, Cc, D, E, score, kfull);
  }
};

__global__ void __launch_bounds__(512) k_t5_count(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_T3];
  const uint32_t lane = lane_id();
  WARP_LOOP(grp, (n + 31) >> 5) {
    const uint32_t t = grp * 32 + lane;
    const bool valid = t < n;
    uint32_t s0 = 0, c = 0;
    Circle3 in_t{};  // this lane's T3 (a, b, c): its circle, the inner circle of all its candidates
    if (valid) {
      const uint32_t m = B.t3_c[t];
      s0 = B.t3_off[m];
      c = B.t3_off[m + 1] - s0;
      if (c) {
        const uint4 abc = B.t3_md4[t];
        in_t = circle3(md_point(B, abc.x), md_point(B, abc.y), md_point(B, abc.z));
      }
    }
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t start = incl - c;  // this lane's T3: candidates [start, incl)
    uint32_t run = 0, bits = 0;
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t t2 = __shfl_sync(FULL, s0, o) + (cc - __shfl_sync(FULL, start, o));
      Circle3 in;  // the owner's inner circle
      in.k = __shfl_sync(FULL, in_t.k, o);
      in.tol = __shfl_sync(FULL, in_t.tol, o);
      bool pass = false;
      if (cand < total) {
        const uint4 abc = B.t3_md4[grp * 32 + o];
        const PointTol Cc = md_point(B, abc.z), D = md_point(B, B.t3_b[t2]), E = md_point(B, B.t3_c[t2]);
        if (t5_in_out_agree(C, in, circle3(Cc, D, E)))
          pass = t5_accept_rest(C, md_point(B, abc.x), md_point(B, abc.y), Cc, D, E);
      }
      const uint32_t bal = __ballot_sync(FULL, pass);
      const uint32_t lo = start > t0 ? min(start - t0, 32u) : 0u;
      const uint32_t hi = incl > t0 ? min(incl - t0, 32u) : 0u;
      if (hi > lo) {
        const uint32_t mine = (bal & (hi == 32u ? FULL : (1u << hi) - 1u)) >> lo;
        run += __popc(mine);
        const uint32_t first = t0 + lo - start;
        if (first < 32u) bits |= mine << first;
      }
    }
    if (valid) {
      B.t5_tcnt[t] = run;
      B.t5_mask[t] = bits;
    }
  }
}


// Count pass with the learned selection.  Only the candidates passing the radius and r-z
// conditions (typically a third of a warp's lanes) need the network, so their inputs go into
// a per-warp queue in shared memory (T5_QCAP entries: inputs, owner lane, position among the
// owner's candidates) and the network runs 32 queued candidates at a time on full warps;
// passes are tallied per owner in shared memory (count, bits of the first 32 candidates).
// Dynamic shared memory: the staged weights, then one queue per warp.
constexpr uint32_t T5_QCAP = 64;  // a chunk adds at most 32 to fewer than 32 waiting
constexpr size_t T5_QWORDS = (T5_NF + 1) * T5_QCAP + 2 * 32;  // per warp: inputs, tags, run, bits
size_t t5_count_mlp_smem(uint32_t block) {
  return (T5_SMEM_FLOATS + (block / 32) * T5_QWORDS) * sizeof(uint32_t);
}

__device__ __forceinline__ void t5_net_drain(const float* Ws, float* qf, const uint32_t* qtag, uint32_t* srun,
                                             uint32_t* sbits, uint32_t head, uint32_t m, uint32_t lane) {
  if (lane < m) {
    const uint32_t slot = (head + lane) & (T5_QCAP - 1);
    float f[T5_NF];
#pragma unroll
    for (int i = 0; i < T5_NF; i++) f[i] = qf[i * T5_QCAP + slot];
    if (t5_mlp_logit(Ws, f) > 0.0f) {
      const uint32_t tag = qtag[slot], o = tag & 31u, k = tag >> 5;
      atomicAdd(&srun[o], 1u);
      if (k < 32u) atomicOr(&sbits[o], 1u << k);
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(512) k_t5_count_mlp(MethodConst C, GeoView G, BufView B,
                                                      const __grid_constant__ T5Mlp M) {
  extern __shared__ __align__(16) uint32_t t5q[];
  float* Ws = reinterpret_cast<float*>(t5q);
  t5_mlp_stage(M, Ws);
  __syncthreads();
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_T3];
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t* wq = t5q + T5_SMEM_FLOATS + (threadIdx.x >> 5) * T5_QWORDS;
  float* qf = reinterpret_cast<float*>(wq);
  uint32_t* qtag = wq + T5_NF * T5_QCAP;
  uint32_t* srun = qtag + T5_QCAP;
  uint32_t* sbits = srun + 32;
  WARP_LOOP(grp, (n + 31) >> 5) {
    const uint32_t t = grp * 32 + lane;
    const bool valid = t < n;
    uint32_t s0 = 0, c = 0;
    if (valid) {
      const uint32_t m = B.t3_c[t];
      s0 = B.t3_off[m];
      c = B.t3_off[m + 1] - s0;
    }
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t start = incl - c;
    srun[lane] = 0u;
    sbits[lane] = 0u;
    __syncwarp();
    uint32_t head = 0, queued = 0;  // warp-uniform
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t so = __shfl_sync(FULL, start, o);
      const uint32_t t2 = __shfl_sync(FULL, s0, o) + (cc - so);
      bool need = false;
      float f[T5_NF];
      if (cand < total) {
        const uint4 abc = B.t3_md4[grp * 32 + o];
        float score, kfull;
        need = t5_mlp_inputs(C, md_point(B, abc.x), md_point(B, abc.y), md_point(B, abc.z), md_point(B, B.t3_b[t2]),
                             md_point(B, B.t3_c[t2]), f, score, kfull);
      }
      const uint32_t bal = __ballot_sync(FULL, need);
      if (need) {
        const uint32_t slot = (head + queued + __popc(bal & lt)) & (T5_QCAP - 1);
#pragma unroll
        for (int i = 0; i < T5_NF; i++) qf[i * T5_QCAP + slot] = f[i];
        qtag[slot] = o | ((cand - so) << 5);
      }
      queued += __popc(bal);
      __syncwarp();
      if (queued >= 32u) {
        t5_net_drain(Ws, qf, qtag, srun, sbits, head, 32u, lane);
        head = (head + 32u) & (T5_QCAP - 1);
        queued -= 32u;
      }
    }
    if (queued) t5_net_drain(Ws, qf, qtag, srun, sbits, head, queued, lane);
    if (valid) {
      B.t5_tcnt[t] = srun[lane];
      B.t5_mask[t] = sbits[lane];
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void t5_emit(const MethodConst& C, const BufView& B, uint32_t k, uint32_t a, uint32_t b,
                                        uint32_t c, uint32_t d, uint32_t e, float score, float kfull) {
  B.t5_m0[k] = a;
  B.t5_m1[k] = b;
  B.t5_m2[k] = c;
  B.t5_m3[k] = d;
  B.t5_m4[k] = e;
  B.t5_md8[2 * (size_t)k] = make_uint4(a, b, c, d);
  B.t5_md8[2 * (size_t)k + 1] = make_uint4(e, 0u, 0u, 0u);
  B.t5_score[k] = score;
  B.t5_kfull[k] = kfull;
}

// Fill pass: passes of T3s with at most 32 candidates come from the stored bits (the score
// and curvature of each are computed once), the others are tested again.  Also writes the
// T5s starting at each MD a, t5_off[a] = t5_toff[t3_off[a]], and zeroes the per-MD counts
// of the duplicate-removal lists (untouched until then).
template <class Sel>
__device__ __forceinline__ void t5_fill_body(const MethodConst& C, const BufView& B, const Sel& sel) {
  const Hdr* H = B.hdr;
  if (H->err) return;
  THREAD_LOOP(a, H->tot[T_MD] + 1) {
    B.t5_off[a] = B.t5_toff[B.t3_off[a]];
    B.c5_cnt[a] = 0u;
    B.c3_cnt[a] = 0u;
    B.ct_cnt[a] = 0u;
  }
  const uint32_t n = H->tot[T_T3];
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  WARP_LOOP(grp, (n + 31) >> 5) {
    const uint32_t t = grp * 32 + lane;
    uint32_t base = 0, np = 0, s0 = 0, c = 0, bits = 0;
    if (t < n) {
      base = B.t5_toff[t];
      np = B.t5_toff[t + 1] - base;
      if (np) {
        const uint32_t m = B.t3_c[t];
        s0 = B.t3_off[m];
        c = B.t3_off[m + 1] - s0;
        bits = B.t5_mask[t];
      }
    }
    const bool small = c <= 32u;
    const uint32_t ns = small ? np : 0u;
    const uint32_t incl = warp_incl_scan(ns);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t k = cc - (__shfl_sync(FULL, incl, o) - __shfl_sync(FULL, ns, o));
      uint32_t m = __shfl_sync(FULL, bits, o);
      const uint32_t s0o = __shfl_sync(FULL, s0, o);
      const uint32_t baseo = __shfl_sync(FULL, base, o);
      if (cand < total) {
        for (uint32_t i = 0; i < k; i++) m &= m - 1u;
        const uint32_t t2 = s0o + (uint32_t)(__ffs(m) - 1);
        const uint4 abc = B.t3_md4[grp * 32 + o];
        const uint32_t d = B.t3_b[t2], e = B.t3_c[t2];
        float score, kfull;
        sel.measure(C, md_point(B, abc.x), md_point(B, abc.y), md_point(B, abc.z), md_point(B, d), md_point(B, e),
                    score, kfull);
        t5_emit(C, B, baseo + k, abc.x, abc.y, abc.z, d, e, score, kfull);
      }
    }
    // T3s with more than 32 candidates: test again, one T3 at a time
    for (uint32_t big = __ballot_sync(FULL, np && !small); big; big &= big - 1u) {
      const uint32_t kk = __ffs(big) - 1;
      const uint32_t ck = __shfl_sync(FULL, c, kk), sk = __shfl_sync(FULL, s0, kk);
      const uint32_t basek = __shfl_sync(FULL, base, kk);
      const uint4 abc = B.t3_md4[grp * 32 + kk];
      const PointTol pa = md_point(B, abc.x), pb = md_point(B, abc.y), pc = md_point(B, abc.z);
      uint32_t run = 0;
      for (uint32_t t0 = 0; t0 < ck; t0 += 32) {
        const uint32_t t2 = sk + t0 + lane;
        float score = 0.0f, kfull = 0.0f;
        uint32_t d = 0, e = 0;
        bool pass = false;
        if (t0 + lane < ck) {
          d = B.t3_b[t2];
          e = B.t3_c[t2];
          pass = sel.select(C, pa, pb, pc, md_point(B, d), md_point(B, e), score, kfull);
        }
        const uint32_t bal = __ballot_sync(FULL, pass);
        if (pass) t5_emit(C, B, basek + run + __popc(bal & lt), abc.x, abc.y, abc.z, d, e, score, kfull);
        run += __popc(bal);
      }
    }
  }
}

__global__ void __launch_bounds__(512) k_t5_fill(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  t5_fill_body(C, B, T5Cuts{});
}

__global__ void __launch_bounds__(512) k_t5_fill_mlp(MethodConst C, GeoView G, BufView B,
                                                     const __grid_constant__ T5Mlp M) {
  __shared__ __align__(16) float Ws[T5_SMEM_FLOATS];
  t5_mlp_stage(M, Ws);
  __syncthreads();
  pdl_wait();
  t5_fill_body(C, B, T5Net{Ws});
}

// ------------------------------------------------------------------ pLS module lookup
__device__ __forceinline__ bool in_sector(const GeoView& G, uint32_t id, float px, float py) {
  const float4 e = G.mod_e[id];
  const float c0 = e.x * py - e.y * px;
  const float c1 = e.z * py - e.w * px;
  return c0 >= 0.0f && c1 < 0.0f;
}

__device__ int find_sector(const GeoView& G, uint32_t row, float px, float py) {
  const uint32_t nphi = G.row_nphi[row], base = G.row_mod_base[row];
  if (G.row_fast[row]) {
    const float two_pi = 6.28318531f;
    float a = atan2f(py, px) - G.row_phi0[row];
    a = a - two_pi * floorf(a / two_pi);
    int k0 = (int)(a * (float)nphi / two_pi);
    k0 = k0 < 0 ? 0 : (k0 >= (int)nphi ? (int)nphi - 1 : k0);
    for (int d = 0; d < 3; d++) {
      const int kk = ((k0 + (d == 0 ? 0 : (d == 1 ? -1 : 1))) % (int)nphi + (int)nphi) % (int)nphi;
      if (in_sector(G, G.row_mods[base + kk], px, py)) return kk;
    }
  }
  for (uint32_t k = 0; k < nphi; k++) {
    const uint32_t id = G.row_mods[base + k];
    if (id == NONE) continue;
    const float4 e = G.mod_e[id];
    const float c0 = e.x * py - e.y * px;
    const float c1 = e.z * py - e.w * px;
    if (c0 >= 0.0f && c1 < 0.0f) return (int)k;
  }
  return -1;
}

__device__ __forceinline__ uint32_t row0_module(const GeoView& G, int s) {
  if (G.surf_nrows[s] == 0) return NONE;
  const uint32_t r = G.surf_row_base[s];
  if (G.row_nphi[r] == 0) return NONE;
  return G.row_mods[G.row_mod_base[r]];
}

// The point where the helix of h first meets surface `which` (0, 1: barrel layers 1, 2;
// 2, 3: the first two disks on its pz side) and the row index of that point on the
// surface; false when it does not meet the surface within the rows (+- 2 rows of margin).
__device__ __forceinline__ bool pls_surface_point(const MethodConst& C, const GeoView& G, const PlsHelix& h,
                                                  int which, int& sf, float& Px, float& Py, int& irow) {
  if (which < 2) {
    sf = which;
    if (G.surf_nrows[sf] == 0) return false;
    const float rl = G.mod_g[G.surf_first[sf]].x;
    const float d2 = h.cx * h.cx + h.cy * h.cy;
    const float d = sqrtf(d2);
    const float a = (rl * rl - h.R * h.R + d2) / (2.0f * d);
    const float h2 = rl * rl - a * a;
    if (!(h2 >= 0.0f)) return false;
    const float hh = sqrtf(h2);
    const float ex = h.cx / d, ey = h.cy / d;
    const float P1x = a * ex - hh * ey, P1y = a * ey + hh * ex;
    const float P2x = a * ex + hh * ey, P2y = a * ey - hh * ex;
    const float wx = h.x0 - h.cx, wy = h.y0 - h.cy;
    const float cr1 = wx * (P1y - h.cy) - wy * (P1x - h.cx);
    const float cr2 = wx * (P2y - h.cy) - wy * (P2x - h.cx);
    const bool f1 = -h.q * cr1 > 0.0f;
    const bool f2 = -h.q * cr2 > 0.0f;
    const float dt1 = wx * (P1x - h.cx) + wy * (P1y - h.cy);
    const float dt2 = wx * (P2x - h.cx) + wy * (P2y - h.cy);
    if (f1 && f2) {
      if (dt1 >= dt2) { Px = P1x; Py = P1y; } else { Px = P2x; Py = P2y; }
    } else if (f1) {
      Px = P1x; Py = P1y;
    } else if (f2) {
      Px = P2x; Py = P2y;
    } else {
      return false;
    }
    const float dxc = Px - h.x0, dyc = Py - h.y0;
    const float chord = sqrtf(dxc * dxc + dyc * dyc);
    const float sarc = arc_length(chord, h.R);
    const float zP = h.z0 + sarc * h.cot;
    const uint32_t m0 = row0_module(G, sf);
    if (m0 == NONE) return false;
    const float4 g0 = G.mod_g[m0];
    const float zlen = g0.w - g0.z;
    const float zhi = g0.z + (float)G.surf_nrows[sf] * zlen;
    if (!(zP > g0.z - 2.0f * zlen && zP < zhi + 2.0f * zlen)) return false;
    irow = (int)floorf((zP - g0.z) / zlen);
    return true;
  }
  if (h.cot == 0.0f) return false;
  sf = (h.cot > 0.0f ? 11 : 6) + (which - 2);
  const uint32_t m0 = row0_module(G, sf);
  if (m0 == NONE) return false;
  const float4 g0 = G.mod_g[m0];
  const float zd = g0.x;
  const float sarc = (zd - h.z0) / h.cot;
  if (!(sarc > 0.0f)) return false;
  const float alpha = sarc / h.R;
  if (!(alpha < C.PI)) return false;
  float sa, ca;
  sin_cos_series(alpha, sa, ca);
  const float sn = -h.q * sa;
  const float wx = h.x0 - h.cx, wy = h.y0 - h.cy;
  Px = h.cx + (wx * ca - wy * sn);
  Py = h.cy + (wx * sn + wy * ca);
  const float rP = sqrtf(Px * Px + Py * Py);
  const float rlen = g0.w - g0.z;
  const float rhi = g0.z + (float)G.surf_nrows[sf] * rlen;
  if (!(rP > g0.z - 2.0f * rlen && rP < rhi + 2.0f * rlen)) return false;
  irow = (int)floorf((rP - g0.z) / rlen);
  return true;
}

// pLS preparation (Sec. 1: pLSs join T3s and T5s) in two launches.  k_pls_prep: one thread
// per (pLS p, r < 12), r = 3 w + d: the helix of p, the point where it first meets surface w
// (barrel layers 1, 2; the first two disks on its pz side) and the modules of sector k - 1,
// k, k + 1 (k the sector of that point) in row (crossing row + d - 1), written to slots
// 3 r .. 3 r + 2 of p's 36 (NONE where there is none); thread r = 0 also stores the helix.
// k_pls_sort: one warp per pLS sorts the 36 slots and drops repeats, which leaves the
// ascending set of distinct candidate module ids.
__global__ void k_pls_prep(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_pls;
  THREAD_LOOP(item, 12u * n) {
    const uint32_t p = item / 12u, r = item - 12u * p;
    uint32_t* slot = B.pls_cand + (size_t)p * MAX_CAND + 3u * r;
    const PlsIn s = H->pls[p];
    if (r == 0) B.pls_ev[p] = find_slot(H->pls_off, H->n_ev, p);
    bool bad = !(isfinite(s.px) && isfinite(s.py) && isfinite(s.pz) && isfinite(s.x0) && isfinite(s.y0) &&
                 isfinite(s.z0)) ||
               (s.charge != 1 && s.charge != -1) || (s.n_hits != 0 && s.n_hits != 3 && s.n_hits != 4);
    PlsHelix h;
    h.pt = sqrtf(s.px * s.px + s.py * s.py);
    if (!(h.pt > 0.0f)) bad = true;
    uint32_t v[3] = {NONE, NONE, NONE};
    if (bad) {
      if (r == 0) atomicOr(&H->err, ERR_BAD_INPUT);
    } else {
      h.R = h.pt / C.KB;
      const float ux = s.px / h.pt;
      const float uy = s.py / h.pt;
      h.q = (float)s.charge;
      const float qR = h.q * h.R;
      h.x0 = s.x0; h.y0 = s.y0; h.z0 = s.z0;
      h.cx = s.x0 + qR * uy;
      h.cy = s.y0 - qR * ux;
      h.cot = s.pz / h.pt;
      if (r == 0) {
        B.pls_h0[p] = make_float4(h.x0, h.y0, h.z0, h.R);
        B.pls_h1[p] = make_float4(h.cx, h.cy, h.cot, h.q);
        B.pls_pt[p] = h.pt;
      }
      int sf, irow;
      float Px, Py;
      if (pls_surface_point(C, G, h, (int)(r / 3), sf, Px, Py, irow)) {
        const int row = irow + (int)(r % 3) - 1;
        if (row >= 0 && (uint32_t)row < G.surf_nrows[sf]) {
          const uint32_t rr = G.surf_row_base[sf] + (uint32_t)row;
          if (G.row_nphi[rr] != 0) {
            const int k = find_sector(G, rr, Px, Py);
            if (k >= 0) {
              const int nphi = (int)G.row_nphi[rr];
#pragma unroll
              for (int d = -1; d <= 1; d++) v[d + 1] = G.row_mods[G.row_mod_base[rr] + ((k + d) % nphi + nphi) % nphi];
            }
          }
        }
      }
    }
    slot[0] = v[0];
    slot[1] = v[1];
    slot[2] = v[2];
  }
}

__global__ void k_pls_sort(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_pls;
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  WARP_LOOP(p, n) {
    uint32_t* slots = B.pls_cand + (size_t)p * MAX_CAND;
    // 36 slots in 64: slot i in lane i (a) or lane i - 32 (b)
    uint32_t a = slots[lane];
    uint32_t b = lane < MAX_CAND - 32 ? slots[32 + lane] : NONE;
#pragma unroll
    for (uint32_t k = 2; k <= 64; k <<= 1) {
#pragma unroll
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        if (j == 32) {  // partners lane, lane + 32 in the same lane; k == 64: ascending
          const uint32_t lo = min(a, b), hi = max(a, b);
          a = lo;
          b = hi;
        } else {
          const uint32_t pa = __shfl_xor_sync(FULL, a, j), pb = __shfl_xor_sync(FULL, b, j);
          const bool lower = (lane & j) == 0;
          const bool asc_a = (lane & k) == 0, asc_b = ((lane + 32) & k) == 0;
          a = (lower == asc_a) ? min(a, pa) : max(a, pa);
          b = (lower == asc_b) ? min(b, pb) : max(b, pb);
        }
      }
    }
    const uint32_t prev_a = __shfl_up_sync(FULL, a, 1);
    const uint32_t prev_b0 = __shfl_up_sync(FULL, b, 1);
    const uint32_t last_a = __shfl_sync(FULL, a, 31);
    const uint32_t prev_b = lane == 0 ? last_a : prev_b0;
    const bool keep_a = a != NONE && (lane == 0 || a != prev_a);
    const bool keep_b = b != NONE && b != prev_b;
    const uint32_t ba = __ballot_sync(FULL, keep_a), bb = __ballot_sync(FULL, keep_b);
    // every lane has read its slots (the shuffles above): the sorted ids go in place
    if (keep_a) slots[__popc(ba & lt)] = a;
    if (keep_b) slots[__popc(ba) + __popc(bb & lt)] = b;
    if (lane == 0) B.pls_ncand[p] = __popc(ba) + __popc(bb);
  }
}

__device__ __forceinline__ PlsHelix load_helix(const BufView& B, uint32_t p) {
  const float4 a = B.pls_h0[p], b = B.pls_h1[p];
  PlsHelix h;
  h.x0 = a.x; h.y0 = a.y; h.z0 = a.z; h.R = a.w;
  h.cx = b.x; h.cy = b.y; h.cot = b.z; h.q = b.w;
  h.pt = B.pls_pt[p];
  return h;
}

// MD tuples of a T5 and a T3, from their array-of-structs copies.
__device__ __forceinline__ void t5_mds(const BufView& B, uint32_t t, uint32_t m[5]) {
  const uint4 p = B.t5_md8[2 * (size_t)t];
  m[0] = p.x; m[1] = p.y; m[2] = p.z; m[3] = p.w; m[4] = B.t5_md8[2 * (size_t)t + 1].x;
}
__device__ __forceinline__ void t3_mds(const BufView& B, uint32_t t, uint32_t m[3]) {
  const uint4 p = B.t3_md4[t];
  m[0] = p.x; m[1] = p.y; m[2] = p.z;
}

// ------------------------------------------------------------------ pT3 / pT5
constexpr uint32_t PT3_RING = 64;    // queued pre-rejection survivors per warp (> 31 + 32)

// Per unit (event, module): the bounding box of its MDs' lower hits, (x0, x1, y0, y1) and
// (z0, z1, -, -), for pT3 phase 1's module-level pruning.  An empty unit's box is unused.
__global__ void k_md_box(GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  THREAD_LOOP(u, H->n_ev * G.nm) {
    float x0 = 3.0e38f, x1 = -3.0e38f, y0 = 3.0e38f, y1 = -3.0e38f, z0 = 3.0e38f, z1 = -3.0e38f;
    for (uint32_t m = B.md_off[u]; m < B.md_off[u + 1]; m++) {
      const float4 p = B.md_pt[2 * (size_t)m];
      x0 = fminf(x0, p.x);
      x1 = fmaxf(x1, p.x);
      y0 = fminf(y0, p.y);
      y1 = fmaxf(y1, p.y);
      z0 = fminf(z0, p.z);
      z1 = fmaxf(z1, p.z);
    }
    B.md_box[2 * (size_t)u] = make_float4(x0, x1, y0, y1);
    B.md_box[2 * (size_t)u + 1] = make_float4(z0, z1, 0.0f, 0.0f);
  }
}

// Can an MD whose lower hit lies in box (bxy: x0, x1, y0, y1; bz: z0, z1) on a module with
// tolerances t pass pls_anchor_accept for helix h?  Both of its windows are bounded over
// the box: the arc length s from the reference point lies in [chord_min, 1.6 chord_max]
// (s >= chord, and s <= 1.6 chord up to half a turn), so the r-phi window is at most its
// value at 1.6 chord_max and the r-z window at most its value at that s; the r-phi
// residual is at least the distance between the circle and the box, and the r-z residual
// at least the distance between the box's z range and z0 + s cot over that s range.  A
// false answer is certain: the margins (1 % plus 2e-2 cm plus 4e-6 of the lengths
// involved) exceed the float rounding of both sides.
__device__ __forceinline__ bool pls_module_maybe(const MethodConst& C, const PlsHelix& h, const float4& bxy,
                                                 const float4& bz, const float4& t) {
  // distances from the reference point (chord) and from the circle's centre to the box
  const float px = fmaxf(fmaxf(bxy.x - h.x0, h.x0 - bxy.y), 0.0f), py = fmaxf(fmaxf(bxy.z - h.y0, h.y0 - bxy.w), 0.0f);
  const float ch_lo = sqrtf(px * px + py * py);
  const float fx = fmaxf(fabsf(bxy.x - h.x0), fabsf(bxy.y - h.x0)), fy = fmaxf(fabsf(bxy.z - h.y0), fabsf(bxy.w - h.y0));
  const float ch_hi = sqrtf(fx * fx + fy * fy);
  const float qx = fmaxf(fmaxf(bxy.x - h.cx, h.cx - bxy.y), 0.0f), qy = fmaxf(fmaxf(bxy.z - h.cy, h.cy - bxy.w), 0.0f);
  const float d_lo = sqrtf(qx * qx + qy * qy);
  const float gx = fmaxf(fabsf(bxy.x - h.cx), fabsf(bxy.y - h.cx)), gy = fmaxf(fabsf(bxy.z - h.cy), fabsf(bxy.w - h.cy));
  const float d_hi = sqrtf(gx * gx + gy * gy);
  const float slack = 0.02f + 4.0e-6f * (h.R + d_hi + ch_hi);
  const float s_lo = ch_lo, s_hi = 1.6f * ch_hi;
  const float wphi = C.W0 + 0.003f * s_hi + 0.015f * s_hi * s_hi / h.R + t.y;
  const float rphi = fmaxf(fmaxf(d_lo - h.R, h.R - d_hi), 0.0f);
  if (rphi > wphi * 1.01f + slack) return false;
  const float zp0 = h.z0 + fminf(s_lo * h.cot, s_hi * h.cot), zp1 = h.z0 + fmaxf(s_lo * h.cot, s_hi * h.cot);
  const float rz = fmaxf(fmaxf(bz.x - zp1, zp0 - bz.y), 0.0f);
  const float wz = 0.05f + 0.002f * s_hi + t.x + t.y * fabsf(h.cot);
  return !(rz > wz * 1.01f + slack + 4.0e-6f * (fabsf(h.z0) + fabsf(bz.x) + fabsf(bz.y) + s_hi * fabsf(h.cot)));
}

// pT3 phase 1 (Sec. 1: pLS + T3), on its own so that it can run beside the LS, T3 and T5
// stages (it needs only the MDs and the pLS preparation).  Unit = pLS p, one warp: the
// first-anchor window on every MD of p's candidate modules; a cheap pre-rejection runs on
// every MD, survivors are queued in MD order and the full window test runs on 32 of them
// at a time, so the passing MDs (at most PLS_MD_CAP kept, else NONE) come out in MD order.
__global__ void __launch_bounds__(512) k_pt3_first_anchor(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->n_pls;
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  __shared__ uint32_t pt3_ring[512 / 32][PT3_RING];
  DYN_LOOP(p, &B.hdr->work[W_PT3_FIRST], n, 2) {
    const PlsHelix h = load_helix(B, p);
    const float inv_r = 1.0f / h.R;
    const uint32_t ubase = B.pls_ev[p] * G.nm;
    const uint32_t* cand = B.pls_cand + (size_t)p * MAX_CAND;
    const uint32_t nc = B.pls_ncand[p];
    uint32_t* mlist = B.pls_mdpass + (size_t)p * PLS_MD_CAP;
    uint32_t npass;
    {
      // the pre-rejection runs on every MD; survivors are queued in MD order and the full
      // window test runs on 32 of them at a time, so passes are appended in MD order
      uint32_t* ring = pt3_ring[threadIdx.x >> 5];
      uint32_t qh = 0, qt = 0;
      npass = 0;
      auto accept_queued = [&](uint32_t nq) {
        const uint32_t m = lane < nq ? ring[(qh + lane) & (PT3_RING - 1)] : 0u;
        const bool pass = lane < nq && pls_anchor_accept(C, h, md_point(B, m));
        const uint32_t bal = __ballot_sync(FULL, pass);
        if (pass && npass + __popc(bal & lt) < PLS_MD_CAP) mlist[npass + __popc(bal & lt)] = m;
        npass += __popc(bal);
        qh += nq;
      };
      for (uint32_t g0 = 0; g0 < nc; g0 += 32) {
        uint32_t b = 0, c = 0;
        if (g0 + lane < nc) {
          const uint32_t mod = cand[g0 + lane], u = ubase + mod;
          b = B.md_off[u];
          c = B.md_off[u + 1] - b;
          // a module none of whose MDs can pass the window holds no first anchor
          if (c && !pls_module_maybe(C, h, B.md_box[2 * (size_t)u], B.md_box[2 * (size_t)u + 1], G.modc[mod])) c = 0;
        }
        const uint32_t incl = warp_incl_scan(c);
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        for (uint32_t t0 = 0; t0 < total; t0 += 32) {
          const uint32_t cc0 = t0 + lane;
          const uint32_t cc = cc0 < total ? cc0 : total - 1;
          const uint32_t o = owner_lane(incl, cc);
          const uint32_t bo = __shfl_sync(FULL, b, o);
          const uint32_t co = __shfl_sync(FULL, c, o);
          const uint32_t io = __shfl_sync(FULL, incl, o);
          const uint32_t m = bo + (cc - (io - co));
          const bool maybe = cc0 < total && pls_anchor_maybe_fast(C, h, inv_r, md_point(B, m));
          const uint32_t mb = __ballot_sync(FULL, maybe);
          if (maybe) ring[(qt + __popc(mb & lt)) & (PT3_RING - 1)] = m;
          qt += __popc(mb);
          __syncwarp();
          if (qt - qh >= 32) {
            accept_queued(32);
            __syncwarp();
          }
        }
      }
      if (qt != qh) accept_queued(qt - qh);
      __syncwarp();
      if (npass > PLS_MD_CAP) npass = NONE;
      if (lane == 0) {
        B.pls_nmdpass[p] = npass;
        B.pt3_icnt[p] = npass != NONE ? npass : nc;  // pT3 items of p
      }
      __syncwarp();
    }
  }
}

// pT3 (Sec. 1: pLS + T3).  Phase 1 (k_pt3_first_anchor) tests pLS p against every MD on
// its candidate modules (the first anchor of any T3 it could join) and keeps the passing
// MDs in order; phase 2 tests the other two anchors of the T3s starting at those MDs.  The
// set equals "T3s whose first MD is on a candidate module, all three anchors inside the
// windows" and comes out in T3 order.  More than PLS_MD_CAP passing MDs: the pLS falls back
// to all T3s of its candidate modules, all three anchors tested.  Phase 2 runs over items:
// item k of p is its k-th passing MD (or k-th candidate module in the fallback), with the
// T3s starting there (there) as candidates, so p's pT3s are its items' passes in item order.

// The item -> pLS table, from the items' offsets (scan of pt3_icnt).  One warp per pLS.
__global__ void k_pt3_items(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t lane = lane_id();
  WARP_LOOP(p, H->n_pls) {
    const uint32_t b = B.pt3_ioff[p], c = B.pt3_ioff[p + 1] - b;
    for (uint32_t i = lane; i < c; i += 32) B.pt3_item_p[b + i] = p;
  }
}

// Item x: its pLS p, whether all three anchors are tested, and its T3 range [b, b + c).
__device__ __forceinline__ void pt3_item(const GeoView& G, const BufView& B, uint32_t x, uint32_t& p, bool& full,
                                         uint32_t& b, uint32_t& c) {
  p = B.pt3_item_p[x];
  const uint32_t k = x - B.pt3_ioff[p];
  full = B.pls_nmdpass[p] == NONE;
  if (!full) {
    const uint32_t m = B.pls_mdpass[(size_t)p * PLS_MD_CAP + k];
    b = B.t3_off[m];
    c = B.t3_off[m + 1] - b;
  } else {
    const uint32_t u = B.pls_ev[p] * G.nm + B.pls_cand[(size_t)p * MAX_CAND + k];
    b = B.t3_off[B.md_off[u]];
    c = B.t3_off[B.md_off[u + 1]] - b;
  }
}

__device__ __forceinline__ bool pt3_test(const MethodConst& C, const BufView& B, const PlsHelix& h, bool full,
                                         uint32_t t) {
  if (full && !pls_anchor_accept(C, h, md_point(B, B.t3_a[t]))) return false;
  return pls_anchor_accept(C, h, md_point(B, B.t3_b[t])) && pls_anchor_accept(C, h, md_point(B, B.t3_c[t]));
}

__device__ __forceinline__ float pt3_score(const MethodConst& C, const BufView& B, const PlsHelix& h, uint32_t t) {
  float score = 0.0f;
  pls_anchor(C, h, md_point(B, B.t3_a[t]), score);
  pls_anchor(C, h, md_point(B, B.t3_b[t]), score);
  pls_anchor(C, h, md_point(B, B.t3_c[t]), score);
  return score;
}

// Count pass: a warp takes 32 consecutive items and walks their concatenated candidates 32
// at a time, keeping each item's count and the pass bits of its first 32 candidates.
__global__ void __launch_bounds__(512) k_pt3_count(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_PT3I];
  const uint32_t lane = lane_id();
  DYN_LOOP(grp, &B.hdr->work[W_PT3_COUNT], (n + 31) >> 5, 2) {
    const uint32_t x = grp * 32 + lane;
    const bool valid = x < n;
    uint32_t b = 0, c = 0, p = 0;
    bool full = false;
    if (valid) pt3_item(G, B, x, p, full, b, c);
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t start = incl - c;  // this lane's item: candidates [start, incl)
    uint32_t run = 0, bits = 0;
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t so = __shfl_sync(FULL, start, o);
      const uint32_t bo = __shfl_sync(FULL, b, o);
      const uint32_t po = __shfl_sync(FULL, p, o);
      const bool fo = __shfl_sync(FULL, (uint32_t)full, o) != 0u;
      const bool pass = cand < total && pt3_test(C, B, load_helix(B, po), fo, bo + (cc - so));
      const uint32_t bal = __ballot_sync(FULL, pass);
      const uint32_t lo = start > t0 ? min(start - t0, 32u) : 0u;
      const uint32_t hi = incl > t0 ? min(incl - t0, 32u) : 0u;
      if (hi > lo) {
        const uint32_t mine = (bal & (hi == 32u ? FULL : (1u << hi) - 1u)) >> lo;
        run += __popc(mine);
        const uint32_t first = t0 + lo - start;
        if (first < 32u) bits |= mine << first;
      }
    }
    if (valid) {
      B.pt3_xcnt[x] = run;
      B.pt3_xmask[x] = bits;
    }
  }
}

// Fill pass in item order (coalesced stores): passes of items with at most 32 candidates
// come from the stored bits, the others are tested again; also writes the per-pLS offsets.
__global__ void __launch_bounds__(512) k_pt3_fill(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_PT3I];
  THREAD_LOOP(q, H->n_pls + 1) B.pt3_off[q] = B.pt3_xoff[B.pt3_ioff[q]];
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  WARP_LOOP(grp, (n + 31) >> 5) {
    const uint32_t x = grp * 32 + lane;
    uint32_t base = 0, np = 0, b = 0, c = 0, p = 0, bits = 0;
    bool full = false;
    if (x < n) {
      base = B.pt3_xoff[x];
      np = B.pt3_xoff[x + 1] - base;
      if (np) {
        pt3_item(G, B, x, p, full, b, c);
        bits = B.pt3_xmask[x];
      }
    }
    const bool small = c <= 32u;
    const uint32_t ns = small ? np : 0u;
    const uint32_t incl = warp_incl_scan(ns);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t k = cc - (__shfl_sync(FULL, incl, o) - __shfl_sync(FULL, ns, o));
      uint32_t m = __shfl_sync(FULL, bits, o);
      const uint32_t bo = __shfl_sync(FULL, b, o);
      const uint32_t po = __shfl_sync(FULL, p, o);
      const uint32_t baseo = __shfl_sync(FULL, base, o);
      if (cand < total) {
        for (uint32_t i = 0; i < k; i++) m &= m - 1u;
        const uint32_t t = bo + (uint32_t)(__ffs(m) - 1);
        B.pt3_pls[baseo + k] = po;
        B.pt3_obj[baseo + k] = t;
        B.pt3_score[baseo + k] = pt3_score(C, B, load_helix(B, po), t);
      }
    }
    // items with more than 32 candidates: test again, one item at a time
    for (uint32_t big = __ballot_sync(FULL, np && !small); big; big &= big - 1u) {
      const uint32_t kk = __ffs(big) - 1;
      const uint32_t ck = __shfl_sync(FULL, c, kk), bk = __shfl_sync(FULL, b, kk);
      const uint32_t pk = __shfl_sync(FULL, p, kk), basek = __shfl_sync(FULL, base, kk);
      const bool fk = __shfl_sync(FULL, (uint32_t)full, kk) != 0u;
      const PlsHelix h = load_helix(B, pk);
      uint32_t run = 0;
      for (uint32_t t0 = 0; t0 < ck; t0 += 32) {
        const uint32_t t = bk + t0 + lane;
        const bool pass = t0 + lane < ck && pt3_test(C, B, h, fk, t);
        const uint32_t bal = __ballot_sync(FULL, pass);
        if (pass) {
          const uint32_t pos = basek + run + __popc(bal & lt);
          B.pt3_pls[pos] = pk;
          B.pt3_obj[pos] = t;
          B.pt3_score[pos] = pt3_score(C, B, h, t);
        }
        run += __popc(bal);
      }
    }
  }
}

// pT5 (Sec. 1: pLS + T5).  A pT5 tests the same windows on anchors a, b, c as the pT3 of the
// T5's first T3 (a, b, c), so its candidates are exactly the T5s built on the pT3s of p
// (t5_toff per T3); the other two anchors and the curvature decide.  Items are the pT3s x
// = (pLS p, T3 t), with the T5s built on t as candidates: p's pT5s are its pT3s' passes in
// pT3 order, so per-item counts scanned over the pT3s give every pT5's position, and a pLS
// with many pT3s is spread over many warps.
__device__ __forceinline__ bool pt5_test(const MethodConst& C, const BufView& B, const PlsHelix& h, uint32_t t) {
  uint32_t m[5];
  t5_mds(B, t, m);
  if (!pls_anchor_accept(C, h, md_point(B, m[3]))) return false;
  if (!pls_anchor_accept(C, h, md_point(B, m[4]))) return false;
  const Circle3 fu = circle3(md_point(B, m[0]), md_point(B, m[2]), md_point(B, m[4]));
  return fabsf(fabsf(B.t5_kfull[t]) - 1.0f / h.R) <= C.KPT5 / h.R + fu.tol;
}

// Anchors m0, m1, m2 are the parent pT3's a, b, c, summed in the same order: its score is
// this sum after three terms, bit for bit.
__device__ __forceinline__ float pt5_score(const MethodConst& C, const BufView& B, const PlsHelix& h, uint32_t x,
                                           uint32_t t) {
  float score = B.pt3_score[x];
  pls_anchor(C, h, md_point(B, B.t5_md8[2 * (size_t)t].w), score);
  pls_anchor(C, h, md_point(B, B.t5_md8[2 * (size_t)t + 1].x), score);
  return score;
}

// Count pass: a warp takes 32 consecutive pT3s and walks their concatenated candidates 32
// at a time (as the MD count pass does), keeping each item's count and the pass bits of its
// first 32 candidates.
__global__ void __launch_bounds__(512) k_pt5_count(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_PT3];
  const uint32_t lane = lane_id();
  DYN_LOOP(grp, &B.hdr->work[W_PT5_COUNT], (n + 31) >> 5, 2) {
    const uint32_t x = grp * 32 + lane;
    const bool valid = x < n;
    uint32_t b = 0, c = 0, p = 0;
    if (valid) {
      p = B.pt3_pls[x];
      const uint32_t t = B.pt3_obj[x];
      b = B.t5_toff[t];
      c = B.t5_toff[t + 1] - b;
    }
    const uint32_t incl = warp_incl_scan(c);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint32_t start = incl - c;  // this lane's item: candidates [start, incl)
    uint32_t run = 0, bits = 0;
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t so = __shfl_sync(FULL, start, o);
      const uint32_t bo = __shfl_sync(FULL, b, o);
      const uint32_t po = __shfl_sync(FULL, p, o);
      const bool pass = cand < total && pt5_test(C, B, load_helix(B, po), bo + (cc - so));
      const uint32_t bal = __ballot_sync(FULL, pass);
      const uint32_t lo = start > t0 ? min(start - t0, 32u) : 0u;
      const uint32_t hi = incl > t0 ? min(incl - t0, 32u) : 0u;
      if (hi > lo) {
        const uint32_t mine = (bal & (hi == 32u ? FULL : (1u << hi) - 1u)) >> lo;
        run += __popc(mine);
        const uint32_t first = t0 + lo - start;
        if (first < 32u) bits |= mine << first;
      }
    }
    if (valid) {
      B.pt5_xcnt[x] = run;
      B.pt5_xmask[x] = bits;
    }
  }
}

// Fill pass in pT3 order (coalesced stores): passes of items with at most 32 candidates
// come from the stored bits, the others are tested again; also writes the per-pLS offsets.
__global__ void __launch_bounds__(512) k_pt5_fill(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_PT3];
  THREAD_LOOP(q, H->n_pls + 1) B.pt5_off[q] = B.pt5_xoff[B.pt3_off[q]];
  const uint32_t lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  WARP_LOOP(grp, (n + 31) >> 5) {
    const uint32_t x = grp * 32 + lane;
    uint32_t base = 0, np = 0, b = 0, c = 0, p = 0, bits = 0;
    if (x < n) {
      base = B.pt5_xoff[x];
      np = B.pt5_xoff[x + 1] - base;
      if (np) {
        p = B.pt3_pls[x];
        const uint32_t t = B.pt3_obj[x];
        b = B.t5_toff[t];
        c = B.t5_toff[t + 1] - b;
        bits = B.pt5_xmask[x];
      }
    }
    const bool small = c <= 32u;
    const uint32_t ns = small ? np : 0u;
    const uint32_t incl = warp_incl_scan(ns);
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
      const uint32_t cand = t0 + lane;
      const uint32_t cc = cand < total ? cand : total - 1;
      const uint32_t o = owner_lane(incl, cc);
      const uint32_t k = cc - (__shfl_sync(FULL, incl, o) - __shfl_sync(FULL, ns, o));
      uint32_t m = __shfl_sync(FULL, bits, o);
      const uint32_t bo = __shfl_sync(FULL, b, o);
      const uint32_t po = __shfl_sync(FULL, p, o);
      const uint32_t baseo = __shfl_sync(FULL, base, o);
      if (cand < total) {
        for (uint32_t i = 0; i < k; i++) m &= m - 1u;
        const uint32_t t = bo + (uint32_t)(__ffs(m) - 1);
        const uint32_t xo = grp * 32 + o;
        B.pt5_pls[baseo + k] = po;
        B.pt5_obj[baseo + k] = t;
        B.pt5_score[baseo + k] = pt5_score(C, B, load_helix(B, po), xo, t);
      }
    }
    // items with more than 32 candidates: test again, one item at a time
    for (uint32_t big = __ballot_sync(FULL, np && !small); big; big &= big - 1u) {
      const uint32_t kk = __ffs(big) - 1;
      const uint32_t ck = __shfl_sync(FULL, c, kk), bk = __shfl_sync(FULL, b, kk);
      const uint32_t pk = __shfl_sync(FULL, p, kk), basek = __shfl_sync(FULL, base, kk);
      const uint32_t xk = grp * 32 + kk;
      const PlsHelix h = load_helix(B, pk);
      uint32_t run = 0;
      for (uint32_t t0 = 0; t0 < ck; t0 += 32) {
        const uint32_t t = bk + t0 + lane;
        const bool pass = t0 + lane < ck && pt5_test(C, B, h, t);
        const uint32_t bal = __ballot_sync(FULL, pass);
        if (pass) {
          const uint32_t pos = basek + run + __popc(bal & lt);
          B.pt5_pls[pos] = pk;
          B.pt5_obj[pos] = t;
          B.pt5_score[pos] = pt5_score(C, B, h, xk, t);
        }
        run += __popc(bal);
      }
    }
  }
}

// ------------------------------------------------------------------ duplicate removal
template <int NA, int NB>
__device__ __forceinline__ int shared_mds(const uint32_t (&a)[NA], const uint32_t (&b)[NB]) {
  int c = 0;
#pragma unroll
  for (int i = 0; i < NA; i++)
#pragma unroll
    for (int j = 0; j < NB; j++) c += a[i] == b[j];
  return c;
}
__device__ __forceinline__ bool better(float sy, uint32_t y, float sx, uint32_t x) {
  return sy < sx || (sy == sx && y < x);
}

// MD -> object lists for pT5 (5 MDs each), pT3 (3) and T5 (5).
__global__ void k_csr_count(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n5 = H->tot[T_PT5], n3 = H->tot[T_PT3], nt = H->tot[T_T5];
  THREAD_LOOP(i, n5 + n3 + nt) {
    if (i < n5) {
      uint32_t m[5];
      t5_mds(B, B.pt5_obj[i], m);
      for (int k = 0; k < 5; k++) atomicAdd(&B.c5_cnt[m[k]], 1u);
    } else if (i < n5 + n3) {
      uint32_t m[3];
      t3_mds(B, B.pt3_obj[i - n5], m);
      for (int k = 0; k < 3; k++) atomicAdd(&B.c3_cnt[m[k]], 1u);
    } else {
      uint32_t m[5];
      t5_mds(B, i - n5 - n3, m);
      for (int k = 0; k < 5; k++) atomicAdd(&B.ct_cnt[m[k]], 1u);
    }
  }
}

__global__ void k_csr_fill(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n5 = H->tot[T_PT5], n3 = H->tot[T_PT3], nt = H->tot[T_T5];
  THREAD_LOOP(i, n5 + n3 + nt) {
    if (i < n5) {
      uint32_t m[5];
      t5_mds(B, B.pt5_obj[i], m);
      for (int k = 0; k < 5; k++) B.c5_list[B.c5_off[m[k]] + atomicSub(&B.c5_cnt[m[k]], 1u) - 1u] = i;
    } else if (i < n5 + n3) {
      uint32_t m[3];
      t3_mds(B, B.pt3_obj[i - n5], m);
      for (int k = 0; k < 3; k++) B.c3_list[B.c3_off[m[k]] + atomicSub(&B.c3_cnt[m[k]], 1u) - 1u] = i - n5;
    } else {
      uint32_t m[5];
      const uint32_t x = i - n5 - n3;
      t5_mds(B, x, m);
      for (int k = 0; k < 5; k++) B.ct_list[B.ct_off[m[k]] + atomicSub(&B.ct_cnt[m[k]], 1u) - 1u] = x;
    }
  }
}

// pT5 stage: dies iff a better pT5 shares its pLS or >= 3 MDs.  One warp per pT5: the
// lanes test 32 neighbours at a time (the pLS's other pT5s, then the pT5s on three of its
// MDs -- sharing >= 3 of 5 MDs means sharing one of any three of them).
__global__ void k_kill_pt5(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n = H->tot[T_PT5];
  GROUP_LOOP(x, act, n, KILL_PT5_GROUP) {
    uint32_t p = 0, mx[5] = {0, 0, 0, 0, 0};
    float sx = 0.0f;
    if (act) {
      p = B.pt5_pls[x];
      sx = B.pt5_score[x];
      t5_mds(B, B.pt5_obj[x], mx);
    }
    const bool dead = group_any<KILL_PT5_GROUP>(
        act, 4u,
        [&](uint32_t i, uint32_t& b, uint32_t& c) {
          if (i == 0) {
            b = B.pt5_off[p];
            c = B.pt5_off[p + 1] - b;
          } else {
            const uint32_t m = mx[2 * (i - 1)];
            b = B.c5_off[m];
            c = B.c5_off[m + 1] - b;
          }
        },
        [&](uint32_t i, uint32_t j) {
          const uint32_t y = i == 0 ? j : B.c5_list[j];
          if (y == x || !better(B.pt5_score[y], y, sx, x)) return false;
          if (i == 0) return true;
          uint32_t my[5];
          t5_mds(B, B.pt5_obj[y], my);
          return shared_mds(mx, my) >= 3;
        });
    if (act && (lane_id() & (KILL_PT5_GROUP - 1)) == 0) B.alive5[x] = dead ? 0u : 1u;
  }
}

// Is pLS p used by a surviving pT5?
__device__ __forceinline__ bool pls_used5(const BufView& B, uint32_t p) {
  for (uint32_t y = B.pt5_off[p]; y < B.pt5_off[p + 1]; y++)
    if (B.alive5[y]) return true;
  return false;
}

// pT3 across stages: its pLS is used by a surviving pT5, or it shares >= 2 MDs with one.
__global__ void k_cross_pt3(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  THREAD_LOOP(x, H->tot[T_PT3]) {
    bool dead = pls_used5(B, B.pt3_pls[x]);
    uint32_t mx[3];
    t3_mds(B, B.pt3_obj[x], mx);
    // sharing >= 2 of x's 3 MDs means sharing one of any 2 of them
    for (int k = 0; k < 2 && !dead; k++) {
      const uint32_t m = mx[k];
      for (uint32_t j = B.c5_off[m]; j < B.c5_off[m + 1] && !dead; j++) {
        const uint32_t z = B.c5_list[j];
        if (!B.alive5[z]) continue;
        uint32_t mz[5];
        t5_mds(B, B.pt5_obj[z], mz);
        if (shared_mds(mx, mz) >= 2) dead = true;
      }
    }
    B.cross3[x] = dead ? 1u : 0u;
  }
}

// pT3 stage among those left: dies iff a better one shares its pLS or >= 2 MDs.
__global__ void k_kill_pt3(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  THREAD_LOOP(x, H->tot[T_PT3]) {
    bool dead = B.cross3[x] != 0;
    const uint32_t p = B.pt3_pls[x];
    const float sx = B.pt3_score[x];
    for (uint32_t y = B.pt3_off[p]; y < B.pt3_off[p + 1] && !dead; y++)
      if (y != x && !B.cross3[y] && better(B.pt3_score[y], y, sx, x)) dead = true;
    uint32_t mx[3];
    t3_mds(B, B.pt3_obj[x], mx);
    for (int k = 0; k < 2 && !dead; k++) {  // >= 2 of 3 shared: two lists suffice
      const uint32_t m = mx[k];
      for (uint32_t j = B.c3_off[m]; j < B.c3_off[m + 1] && !dead; j++) {
        const uint32_t y = B.c3_list[j];
        if (y == x || B.cross3[y]) continue;
        uint32_t my[3];
        t3_mds(B, B.pt3_obj[y], my);
        if (shared_mds(mx, my) >= 2 && better(B.pt3_score[y], y, sx, x)) dead = true;
      }
    }
    B.alive3[x] = dead ? 0u : 1u;
  }
}

// T5 across stages: shares >= 3 MDs with a surviving pT5 or pT3 (one of any three of its
// MDs is then shared).  A group of lanes per T5.  Also flags the pLSs that become track
// candidates themselves: those used by no surviving pT5 or pT3.
__global__ void k_cross_t5(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  THREAD_LOOP(p, H->n_pls) {
    bool used = pls_used5(B, p);
    for (uint32_t y = B.pt3_off[p]; y < B.pt3_off[p + 1] && !used; y++) used = B.alive3[y] != 0;
    B.plstc[p] = used ? 0u : 1u;
  }
  GROUP_LOOP(x, act, H->tot[T_T5], CROSS_T5_GROUP) {
    uint32_t mx[5] = {0, 0, 0, 0, 0};
    if (act) t5_mds(B, x, mx);
    const bool dead = group_any<CROSS_T5_GROUP>(
        act, 6u,
        [&](uint32_t i, uint32_t& b, uint32_t& c) {
          const uint32_t m = mx[2 * (i % 3)];
          const uint32_t* off = i < 3 ? B.c5_off : B.c3_off;
          b = off[m];
          c = off[m + 1] - b;
        },
        [&](uint32_t i, uint32_t j) {
          if (i < 3) {
            const uint32_t z = B.c5_list[j];
            if (!B.alive5[z]) return false;
            uint32_t mz[5];
            t5_mds(B, B.pt5_obj[z], mz);
            return shared_mds(mx, mz) >= 3;
          }
          const uint32_t z = B.c3_list[j];
          if (!B.alive3[z]) return false;
          uint32_t mz[3];
          t3_mds(B, B.pt3_obj[z], mz);
          return shared_mds(mx, mz) >= 3;
        });
    if (act && (lane_id() & (CROSS_T5_GROUP - 1)) == 0) B.crosst[x] = dead ? 1u : 0u;
  }
}

// T5 stage among those left: dies iff a better one shares >= 3 MDs.  One warp per T5.
__global__ void k_kill_t5(BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  GROUP_LOOP(x, act, H->tot[T_T5], KILL_T5_GROUP) {
    bool dead = act && B.crosst[x] != 0;
    {
      float sx = 0.0f;
      uint32_t mx[5] = {0, 0, 0, 0, 0};
      if (act && !dead) {
        sx = B.t5_score[x];
        t5_mds(B, x, mx);
      }
      dead = group_any<KILL_T5_GROUP>(
          act && !dead, 3u,
          [&](uint32_t i, uint32_t& b, uint32_t& c) {
            const uint32_t m = mx[2 * i];
            b = B.ct_off[m];
            c = B.ct_off[m + 1] - b;
          },
          [&](uint32_t, uint32_t j) {
            const uint32_t y = B.ct_list[j];
            if (y == x || B.crosst[y] || !better(B.t5_score[y], y, sx, x)) return false;
            uint32_t my[5];
            t5_mds(B, y, my);
            return shared_mds(mx, my) >= 3;
          }) || dead;
    }
    if (act && (lane_id() & (KILL_T5_GROUP - 1)) == 0) B.alivet[x] = dead ? 0u : 1u;
  }
}

// ------------------------------------------------------------------ track candidates
struct EvCounts {
  uint32_t n5, n3, nt, np, b5, b3, bt, bp;  // counts and first object index of the event
};

__device__ __forceinline__ EvCounts ev_counts(const GeoView& G, const BufView& B, const Hdr* H, uint32_t e) {
  EvCounts c;
  const uint32_t p0 = H->pls_off[e], p1 = H->pls_off[e + 1];
  c.b5 = B.pt5_off[p0];
  c.n5 = B.sa5[B.pt5_off[p1]] - B.sa5[c.b5];
  c.b3 = B.pt3_off[p0];
  c.n3 = B.sa3[B.pt3_off[p1]] - B.sa3[c.b3];
  const uint32_t m0 = B.md_off[e * G.nm], m1 = B.md_off[(e + 1) * G.nm];
  c.bt = B.t5_off[m0];
  c.nt = B.sat[B.t5_off[m1]] - B.sat[c.bt];
  c.bp = p0;
  c.np = B.sap[p1] - B.sap[p0];
  return c;
}

__global__ void k_tc_offsets(GeoView G, BufView B) {
  pdl_wait();
  Hdr* H = B.hdr;
  if (H->err) return;
  __shared__ uint32_t sm[33];
  const uint32_t ne = H->n_ev;
  uint32_t carry = 0;
  for (uint32_t e0 = 0; e0 < ne; e0 += blockDim.x) {
    const uint32_t e = e0 + threadIdx.x;
    uint32_t v = 0;
    if (e < ne) {
      const EvCounts c = ev_counts(G, B, H, e);
      v = c.n5 + c.n3 + c.nt + c.np;
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, sm, tot);
    if (e < ne) B.tc_ev_off[e] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    B.tc_ev_off[ne] = carry;
    H->tot[T_TC] = carry;
    if (carry > B.cap_tc) atomicOr(&H->err, 1u << (ERR_OVERFLOW_SHIFT + T_TC));
  }
}

// npix: the seed's pixel hits (4 for a quad, 3 for a triplet, 0 without a seed).
__device__ __forceinline__ void write_tc(lst_tc* tc, uint8_t type, uint32_t obj, uint32_t pls, const uint32_t* mds,
                                         int nmd, const BufView& B, float pt, float score, uint32_t npix) {
  lst_tc r;
  r.type = type;
  r.n_ot = (uint8_t)(2 * nmd);
  r.n_pix = (uint8_t)npix;
  r.pad = 0;
  r.obj = obj;
  r.pls = pls;
  for (int k = 0; k < 10; k++) r.ot[k] = NONE;
  for (int k = 0; k < nmd; k++) {
    r.ot[2 * k] = B.md_lo_idx[mds[k]];
    r.ot[2 * k + 1] = B.md_up_idx[mds[k]];
  }
  for (uint32_t k = 0; k < 4; k++) r.pix[k] = k < npix ? 4 * pls + k : NONE;
  r.pt = pt;
  r.score = score;
  *tc = r;
}

// Pixel hits of seed p (global index): a triplet has three, anything else four.
__device__ __forceinline__ uint32_t seed_hits(const Hdr* H, uint32_t p) { return H->pls[p].n_hits == 3 ? 3u : 4u; }

// Survivors -> track candidates: per event pT5s, pT3s, T5s, then unused pLSs (Sec. 1 list).
__global__ void k_tc_write(MethodConst C, GeoView G, BufView B) {
  pdl_wait();
  const Hdr* H = B.hdr;
  if (H->err) return;
  const uint32_t n5 = H->tot[T_PT5], n3 = H->tot[T_PT3], nt = H->tot[T_T5], np = H->n_pls;
  lst_tc* tc = (lst_tc*)B.tc;
  THREAD_LOOP(i, n5 + n3 + nt + np) {
    if (i < n5) {
      const uint32_t x = i;
      if (!B.alive5[x]) continue;
      const uint32_t p = B.pt5_pls[x], e = B.pls_ev[p];
      const EvCounts c = ev_counts(G, B, H, e);
      const uint32_t pos = B.tc_ev_off[e] + (B.sa5[x] - B.sa5[c.b5]);
      uint32_t m[5];
      t5_mds(B, B.pt5_obj[x], m);
      write_tc(tc + pos, LST_TC_PT5, x - c.b5, p - c.bp, m, 5, B, B.pls_pt[p], B.pt5_score[x], seed_hits(H, p));
    } else if (i < n5 + n3) {
      const uint32_t x = i - n5;
      if (!B.alive3[x]) continue;
      const uint32_t p = B.pt3_pls[x], e = B.pls_ev[p];
      const EvCounts c = ev_counts(G, B, H, e);
      const uint32_t pos = B.tc_ev_off[e] + c.n5 + (B.sa3[x] - B.sa3[c.b3]);
      uint32_t m[3];
      t3_mds(B, B.pt3_obj[x], m);
      write_tc(tc + pos, LST_TC_PT3, x - c.b3, p - c.bp, m, 3, B, B.pls_pt[p], B.pt3_score[x], seed_hits(H, p));
    } else if (i < n5 + n3 + nt) {
      const uint32_t x = i - n5 - n3;
      if (!B.alivet[x]) continue;
      const uint32_t e = B.md_unit[B.t5_m0[x]] / G.nm;
      const EvCounts c = ev_counts(G, B, H, e);
      const uint32_t pos = B.tc_ev_off[e] + c.n5 + c.n3 + (B.sat[x] - B.sat[c.bt]);
      uint32_t m[5];
      t5_mds(B, x, m);
      write_tc(tc + pos, LST_TC_T5, x - c.bt, NONE, m, 5, B, C.KB / fabsf(B.t5_kfull[x]), B.t5_score[x], 0u);
    } else {
      const uint32_t p = i - n5 - n3 - nt;
      if (!B.plstc[p]) continue;
      const uint32_t e = B.pls_ev[p];
      const EvCounts c = ev_counts(G, B, H, e);
      const uint32_t pos = B.tc_ev_off[e] + c.n5 + c.n3 + c.nt + (B.sap[p] - B.sap[c.bp]);
      write_tc(tc + pos, LST_TC_PLS, p - c.bp, p - c.bp, nullptr, 0, B, B.pls_pt[p], 0.0f, seed_hits(H, p));
    }
  }
}

// ------------------------------------------------------------------ host-side enqueue
// Kernel names in launch order (profile mode records one CUDA event after each).
const char* const kKernelNames[] = {
    "zero_sensor_counts", "hits_count", "(unused)", "scan_large", "(unused)", "hits_scatter", "hits_sort",
    "md_count", "md_fill", "ls_count", "ls_fill", "t3_count", "t3_fill", "t5_count", "t5_fill", "pls_prep",
    "pt3_count", "pt3_fill", "pt5_count", "pt5_fill", "(unused)", "md_lists_count", "md_lists_fill",
    "kill_pt5", "(unused)", "cross_pt3", "kill_pt3", "(unused)", "cross_t5", "kill_t5", "tc_offsets", "tc_write",
    "(unused)", "(unused)", "pt3_first_anchor", "pls_sort", "pt3_items", "md_boxes", "scan_small", "(unused)"};
const int kNumKernelNames = sizeof(kKernelNames) / sizeof(kKernelNames[0]);

struct Marker {
  MarkFn fn;
  void* arg;
  int nk;
  void operator()(int name) {
    nk++;
    if (fn) fn(arg, name);
  }
};

// Launches kernel k on stream s allowing programmatic dependent launch: k may be scheduled
// while the previous kernel on s drains, and waits for it in pdl_wait().
template <typename... KArgs, typename... Args>
static void launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// bound: the most elements the array can hold (its buffer's capacity), which picks the
// one-block scan for small arrays when the pipeline is sized for them.
// slot: this scan's own ticket counter and chunk totals in the header (single-pass form).
static void scan(const BufView& B, const Launch& L, cudaStream_t s, const uint32_t* in, uint32_t* out,
                 const uint32_t* nptr, uint32_t mul, int tot, uint32_t cap, uint64_t bound, uint32_t slot, Marker& mk) {
  if (bound <= SCAN_SMALL_MAX) {
    launch(k_scan_small, 1, 1024, 0, s, in, nptr, mul, B.hdr, out, tot, cap);
    mk(38);
    return;
  }
  launch(k_scan_large, (uint32_t)((bound + SCAN_LARGE_CHUNK - 1) / SCAN_LARGE_CHUNK), 1024, 0, s, in, nptr, mul, B, out,
         tot, cap, slot);
  mk(3);
}

// pT3 item offsets and item -> pLS table.  May run on the side stream beside the main
// chain's scans, so its scan has a slot of its own (5).
static void pt3_items(const BufView& B, const Launch& L, cudaStream_t s, Marker& mk) {
  if (B.cap_pls <= SCAN_SMALL_MAX) {
    launch(k_scan_small, 1, 1024, 0, s, B.pt3_icnt, &B.hdr->n_pls, 1, B.hdr, B.pt3_ioff, T_PT3I, 0xFFFFFFFFu);
    mk(38);
  } else {
    launch(k_scan_large, (B.cap_pls + SCAN_LARGE_CHUNK - 1) / SCAN_LARGE_CHUNK, 1024, 0, s, B.pt3_icnt, &B.hdr->n_pls,
           1, B, B.pt3_ioff, T_PT3I, 0xFFFFFFFFu, 5u);
    mk(3);
  }
  launch(k_pt3_items, L.grid, 256, 0, s, B);
  mk(36);
}

static void scan_multi(const BufView& B, const Launch& L, cudaStream_t s, const ScanJobs& J, int n, uint64_t bound,
                       uint32_t slot0, Marker& mk) {
  if (bound <= SCAN_SMALL_MAX) {
    launch(k_scan_small_multi, n, 1024, 0, s, J, B.hdr);
    mk(38);
    return;
  }
  launch(k_scan_large_multi, dim3((uint32_t)((bound + SCAN_LARGE_CHUNK - 1) / SCAN_LARGE_CHUNK), n), 1024, 0, s, J, B,
         slot0);
  mk(3);
}

// Lets the LS count kernel take the shared memory of the largest block (512 threads) on the
// current device; called once per pipeline, outside any stream capture.
cudaError_t configure_kernels() {
  const int bytes = (int)((512 / 32) * ls_warp_words(LS_LIST_MAX) * sizeof(uint32_t));
  return cudaFuncSetAttribute(k_ls_count, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Loads every kernel of the chain on the current device (cudaFuncGetAttributes resolves
// each function, which lazy module loading otherwise defers to its first launch), so that
// later launches allocate nothing for code or module data.
cudaError_t preload_kernels() {
  const void* ks[] = {
      (const void*)k_scan_small, (const void*)k_scan_small_multi,
      (const void*)k_scan_large, (const void*)k_scan_large_multi, (const void*)k_zero, (const void*)k_hits_count, (const void*)k_hits_scatter,
      (const void*)k_hits_sort, (const void*)k_md_count, (const void*)k_md_fill, (const void*)k_ls_fill,
      (const void*)k_ls_count, (const void*)k_t3_count, (const void*)k_t3_fill, (const void*)k_t5_count,
      (const void*)k_t5_fill, (const void*)k_t5_count_mlp, (const void*)k_t5_fill_mlp, (const void*)k_pls_prep, (const void*)k_pls_sort, (const void*)k_md_box,
      (const void*)k_pt3_first_anchor, (const void*)k_pt3_items, (const void*)k_pt3_count, (const void*)k_pt3_fill,
      (const void*)k_pt5_count, (const void*)k_pt5_fill, (const void*)k_csr_count, (const void*)k_csr_fill,
      (const void*)k_kill_pt5, (const void*)k_cross_pt3, (const void*)k_kill_pt3, (const void*)k_cross_t5,
      (const void*)k_kill_t5, (const void*)k_tc_offsets, (const void*)k_tc_write};
  for (const void* k : ks) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Enqueues the whole chain on stream s; returns the number of kernels launched.  mark (may
// be null) is called after every launch with the index of its name in kKernelNames.
int enqueue_pipeline(const MethodConst& C, const GeoView& G, const BufView& B, const Launch& L, cudaStream_t s,
                     MarkFn mark, void* arg, const SideBranch* side) {
  Marker mk{mark, arg, 0};
  Hdr* H = B.hdr;
  const uint32_t g = L.grid, bs = L.block;
  const uint32_t two_nm = 2 * G.nm;
  if (side) {  // the pLS preparation needs only the inputs: run it beside the OT chain
    cudaEventRecord(side->fork, s);
    cudaStreamWaitEvent(side->s, side->fork, 0);
    launch(k_pls_prep, g, 256, 0, side->s, C, G, B);
    mk(15);
    launch(k_pls_sort, g, 128, 0, side->s, B);
    mk(35);
  }
  launch(k_zero, g, 256, 0, s, B.sen_cnt, &H->n_ev, two_nm, 1);
  mk(0);
  launch(k_hits_count, g, 256, 0, s, G, B);
  mk(1);
  scan(B, L, s, B.sen_cnt, B.sen_off, &H->n_ev, two_nm, T_HITS, 0xFFFFFFFFu, (uint64_t)B.cap_ev * two_nm, 0u, mk);
  launch(k_hits_scatter, g, 256, 0, s, G, B);
  mk(5);
  launch(k_hits_sort, g, 256, 0, s, G, B);
  mk(6);
  launch(k_md_count, g, bs, 0, s, C, G, B);
  mk(7);
  scan(B, L, s, B.md_hcnt, B.md_hoff, &H->n_hits, 1, T_MD, B.cap_md, B.cap_hits, 1u, mk);
  launch(k_md_fill, g, bs, 0, s, C, G, B);
  mk(8);
  if (side) {  // pT3 phase 1 needs the MDs and the pLS preparation only
    cudaEventRecord(side->mds, s);
    cudaStreamWaitEvent(side->s, side->mds, 0);
    launch(k_md_box, g, 256, 0, side->s, G, B);
    mk(37);
    launch(k_pt3_first_anchor, g, bs, 0, side->s, C, G, B);
    mk(34);
    pt3_items(B, L, side->s, mk);
    cudaEventRecord(side->join, side->s);
  }
  const uint32_t lcap = L.ls_list_cap;
  const size_t ls_smem = lcap ? (bs / 32) * ls_warp_words(lcap) * sizeof(uint32_t) : 0;
  launch(k_ls_count, g, bs, ls_smem, s, C, G, B, lcap);
  mk(9);
  scan(B, L, s, B.ls_cnt, B.ls_off, &H->tot[T_MD], 1, T_LS, B.cap_ls, B.cap_md, 2u, mk);
  launch(k_ls_fill, g, bs, 0, s, C, G, B);
  mk(10);
  launch(k_t3_count, g, 256, 0, s, C, G, B);
  mk(11);
  scan(B, L, s, B.t3_lcnt, B.t3_loff, &H->tot[T_LS], 1, T_T3, B.cap_t3, B.cap_ls, 3u, mk);
  launch(k_t3_fill, g, 256, 0, s, C, G, B);
  mk(12);
  if (L.t5_mlp)
    launch(k_t5_count_mlp, g, bs, t5_count_mlp_smem(bs), s, C, G, B, *L.t5_mlp);
  else
    launch(k_t5_count, g, bs, 0, s, C, G, B);
  mk(13);
  scan(B, L, s, B.t5_tcnt, B.t5_toff, &H->tot[T_T3], 1, T_T5, B.cap_t5, B.cap_t3, 4u, mk);
  if (L.t5_mlp)
    launch(k_t5_fill_mlp, g, bs, 0, s, C, G, B, *L.t5_mlp);
  else
    launch(k_t5_fill, g, bs, 0, s, C, G, B);
  mk(14);
  if (side) {
    cudaStreamWaitEvent(s, side->join, 0);
  } else {
    launch(k_pls_prep, g, 256, 0, s, C, G, B);
    mk(15);
    launch(k_pls_sort, g, 128, 0, s, B);
    mk(35);
    launch(k_md_box, g, 256, 0, s, G, B);
    mk(37);
    launch(k_pt3_first_anchor, g, bs, 0, s, C, G, B);
    mk(34);
    pt3_items(B, L, s, mk);
  }
  launch(k_pt3_count, g, bs, 0, s, C, G, B);
  mk(16);
  scan(B, L, s, B.pt3_xcnt, B.pt3_xoff, &H->tot[T_PT3I], 1, T_PT3, B.cap_pt3, (uint64_t)B.cap_pls * PLS_ITEMS, 6u, mk);
  launch(k_pt3_fill, g, bs, 0, s, C, G, B);
  mk(17);
  launch(k_pt5_count, g, bs, 0, s, C, G, B);
  mk(18);
  scan(B, L, s, B.pt5_xcnt, B.pt5_xoff, &H->tot[T_PT3], 1, T_PT5, B.cap_pt5, B.cap_pt3, 7u, mk);
  launch(k_pt5_fill, g, bs, 0, s, C, G, B);
  mk(19);
  launch(k_csr_count, g, 256, 0, s, B);
  mk(21);
  {
    ScanJobs J{};
    J.j[0] = {B.c5_cnt, B.c5_off, &H->tot[T_MD], T_C5, 5u * B.cap_pt5};
    J.j[1] = {B.c3_cnt, B.c3_off, &H->tot[T_MD], T_C3, 3u * B.cap_pt3};
    J.j[2] = {B.ct_cnt, B.ct_off, &H->tot[T_MD], T_CT, 5u * B.cap_t5};
    scan_multi(B, L, s, J, 3, B.cap_md, 8u, mk);
  }
  launch(k_csr_fill, g, 256, 0, s, B);
  mk(22);
  launch(k_kill_pt5, g, 256, 0, s, B);
  mk(23);
  launch(k_cross_pt3, g, 256, 0, s, B);
  mk(25);
  launch(k_kill_pt3, g, 256, 0, s, B);
  mk(26);
  launch(k_cross_t5, g, 256, 0, s, B);
  mk(28);
  launch(k_kill_t5, g, 256, 0, s, B);
  mk(29);
  {
    ScanJobs J{};
    J.j[0] = {B.alive5, B.sa5, &H->tot[T_PT5], T_A5, 0xFFFFFFFFu};
    J.j[1] = {B.alive3, B.sa3, &H->tot[T_PT3], T_A3, 0xFFFFFFFFu};
    J.j[2] = {B.alivet, B.sat, &H->tot[T_T5], T_AT, 0xFFFFFFFFu};
    J.j[3] = {B.plstc, B.sap, &H->n_pls, T_AP, 0xFFFFFFFFu};
    scan_multi(B, L, s, J, 4, std::max<uint64_t>(std::max(B.cap_pt5, B.cap_pt3), std::max(B.cap_t5, B.cap_pls)), 11u,
               mk);
  }
  launch(k_tc_offsets, 1, 1024, 0, s, G, B);
  mk(30);
  launch(k_tc_write, g, 256, 0, s, C, G, B);
  mk(31);
  return mk.nk;
}

}  // namespace lst
