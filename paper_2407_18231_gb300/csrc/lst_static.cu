// lst_run_event_static: the per-event chain for small events with every intermediate list
// in one file-scope device array, so the call allocates no memory at all.
//
// Who needs it: callers that may not allocate device memory once they are running --
// for example a host framework whose pooling allocator owns the GPU (an extra cudaMalloc
// would fragment the pool or break its budget), a latency-critical loop that cannot afford
// cudaMalloc's implicit device synchronisation, or a plug-in loaded into a process that
// forbids device allocations after start-up.  They still create a context once (geometry
// and connection map) and pass their own input and output buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/lst.h"
#include "lst_device.cuh"

namespace lst {
int enqueue_pipeline(const MethodConst& C, const GeoView& G, const BufView& B, const Launch& L, cudaStream_t s,
                     MarkFn mark, void* arg, const SideBranch* side = nullptr);
bool ctx_views(lst_ctx* c, GeoView* g, MethodConst* m, Launch* l, int* device, bool* have_map);
void ctx_set_error(lst_ctx* c, const std::string& msg);
cudaError_t preload_kernels();
cudaError_t static_scratch_prepare(int device);
}  // namespace lst

using namespace lst;

namespace {

// Limits of one call (documented in lst.h).
constexpr uint32_t MAX_MODULES = 16384;
constexpr uint32_t MAX_HITS = 8192;
constexpr uint32_t MAX_PLS = 512;
constexpr uint32_t MAX_MD = 8192;
constexpr uint32_t MAX_LS = 32768;
constexpr uint32_t MAX_T3 = 32768;
constexpr uint32_t MAX_T5 = 16384;
constexpr uint32_t MAX_PT3 = 16384;
constexpr uint32_t MAX_PT5 = 16384;
constexpr uint32_t MASK_WORDS = 65536;  // LS partner lists; a fuller event joins again in the fill pass
constexpr size_t SCRATCH_BYTES = size_t(8) << 20;  // every GPU that loads the library holds this until exit
// chunk states per scan slot of the single-pass scans: the largest bound a scan of one call
// is launched with (2 x modules for the hit bins, pLS x items for the pT3 items, ...)
constexpr uint32_t STATIC_SCAN_BOUND =
    std::max({2 * MAX_MODULES, MAX_HITS, MAX_MD, MAX_LS, MAX_T3, MAX_T5, MAX_PT3, MAX_PT5, MAX_PLS * PLS_ITEMS});
constexpr uint32_t STATIC_SCAN_CHUNKS = (STATIC_SCAN_BOUND + SCAN_LARGE_CHUNK - 1) / SCAN_LARGE_CHUNK;

// The scratch.  In host code `g_scratch` is only a stand-in symbol: its device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_dev[MAX_DEVICES] = {};
// per device, the calls made so far: tags the single-pass scans' chunk states (30 bits),
// which the zero-initialised array holds from earlier calls
uint32_t g_scan_epoch[MAX_DEVICES] = {};

// Sinks for carve_layout: Sizer only adds up the 256-byte aligned extents (usable in a
// constant expression), Placer also points every list into the scratch.
struct Sizer {
  size_t off = 0;
  template <typename T>
  constexpr void take(T*&, size_t n) {
    off = (off + 255) & ~size_t(255);
    off += n * sizeof(T);
  }
};
struct Placer {
  char* base;
  size_t off = 0;
  template <typename T>
  void take(T*& p, size_t n) {
    off = (off + 255) & ~size_t(255);
    p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
  }
};

// Lays every list of one event out in the scratch (through sink c); returns the bytes used.
template <typename Sink>
constexpr size_t carve_layout(Sink& c, BufView& B) {
  c.take(B.hdr, 1);
  B.cap_ev = 1; B.cap_hits = MAX_HITS; B.cap_md = MAX_MD; B.cap_ls = MAX_LS; B.cap_t3 = MAX_T3;
  B.cap_t5 = MAX_T5; B.cap_pls = MAX_PLS; B.cap_pt3 = MAX_PT3; B.cap_pt5 = MAX_PT5;
  c.take(B.sen_cnt, 2 * MAX_MODULES + 1);
  c.take(B.sen_off, 2 * MAX_MODULES + 1);
  c.take(B.hit_tmp, MAX_HITS);
  c.take(B.hit_psi, MAX_HITS);
  c.take(B.hit_ev, MAX_HITS);
  c.take(B.hit_idx, MAX_HITS);
  c.take(B.hit4, MAX_HITS);
  c.take(B.hit_sen, MAX_HITS);
  c.take(B.md_hcnt, MAX_HITS);
  c.take(B.md_hoff, MAX_HITS + 1);
  c.take(B.md_hmask, MAX_HITS);
  c.take(B.md_off, MAX_MODULES + 1);
  c.take(B.md_box, 2 * (size_t)MAX_MODULES);
  c.take(B.md_unit, MAX_MD);
  c.take(B.md_lo_idx, MAX_MD);
  c.take(B.md_up_idx, MAX_MD);
  c.take(B.md_pt, 2 * MAX_MD);
  c.take(B.md_up4, MAX_MD);
  c.take(B.md_dir4, MAX_MD);
  c.take(B.md_psi, MAX_MD);
  c.take(B.ls_cnt, MAX_MD);
  c.take(B.ls_off, MAX_MD + 1);
  c.take(B.ls_in, MAX_LS);
  c.take(B.ls_out, MAX_LS);
  c.take(B.t3_lcnt, MAX_LS);
  c.take(B.t3_mask, MAX_LS);
  c.take(B.t3_loff, MAX_LS + 1);
  c.take(B.t3_off, MAX_MD + 1);
  c.take(B.t3_a, MAX_T3);
  c.take(B.t3_b, MAX_T3);
  c.take(B.t3_c, MAX_T3);
  c.take(B.t3_md4, MAX_T3);
  c.take(B.t5_tcnt, MAX_T3);
  c.take(B.t5_mask, MAX_T3);
  c.take(B.t5_toff, MAX_T3 + 1);
  c.take(B.t5_off, MAX_MD + 1);
  c.take(B.t5_m0, MAX_T5);
  c.take(B.t5_m1, MAX_T5);
  c.take(B.t5_m2, MAX_T5);
  c.take(B.t5_m3, MAX_T5);
  c.take(B.t5_m4, MAX_T5);
  c.take(B.t5_score, MAX_T5);
  c.take(B.t5_kfull, MAX_T5);
  c.take(B.t5_md8, 2 * MAX_T5);
  c.take(B.pls_ev, MAX_PLS);
  c.take(B.pls_ncand, MAX_PLS);
  c.take(B.pls_cand, (size_t)MAX_PLS * MAX_CAND);
  c.take(B.pls_mdpass, (size_t)MAX_PLS * PLS_MD_CAP);
  c.take(B.pls_nmdpass, MAX_PLS);
  c.take(B.pls_h0, MAX_PLS);
  c.take(B.pls_h1, MAX_PLS);
  c.take(B.pls_pt, MAX_PLS);
  c.take(B.pt3_icnt, MAX_PLS);
  c.take(B.pt3_ioff, MAX_PLS + 1);
  c.take(B.pt3_item_p, (size_t)MAX_PLS * PLS_ITEMS);
  c.take(B.pt3_xcnt, (size_t)MAX_PLS * PLS_ITEMS);
  c.take(B.pt3_xoff, (size_t)MAX_PLS * PLS_ITEMS + 1);
  c.take(B.pt3_xmask, (size_t)MAX_PLS * PLS_ITEMS);
  c.take(B.pt3_off, MAX_PLS + 1);
  c.take(B.pt3_pls, MAX_PT3);
  c.take(B.pt3_obj, MAX_PT3);
  c.take(B.pt3_score, MAX_PT3);
  c.take(B.pt5_xcnt, MAX_PT3);
  c.take(B.pt5_xoff, MAX_PT3 + 1);
  c.take(B.pt5_xmask, MAX_PT3);
  c.take(B.pt5_off, MAX_PLS + 1);
  c.take(B.pt5_pls, MAX_PT5);
  c.take(B.pt5_obj, MAX_PT5);
  c.take(B.pt5_score, MAX_PT5);
  c.take(B.c5_cnt, MAX_MD + 1);
  c.take(B.c5_off, MAX_MD + 1);
  c.take(B.c5_list, (size_t)5 * MAX_PT5);
  c.take(B.c3_cnt, MAX_MD + 1);
  c.take(B.c3_off, MAX_MD + 1);
  c.take(B.c3_list, (size_t)3 * MAX_PT3);
  c.take(B.ct_cnt, MAX_MD + 1);
  c.take(B.ct_off, MAX_MD + 1);
  c.take(B.ct_list, (size_t)5 * MAX_T5);
  c.take(B.alive5, MAX_PT5);
  c.take(B.alive3, MAX_PT3);
  c.take(B.alivet, MAX_T5);
  c.take(B.plstc, MAX_PLS);
  c.take(B.cross3, MAX_PT3);
  c.take(B.crosst, MAX_T5);
  c.take(B.sa5, MAX_PT5 + 1);
  c.take(B.sa3, MAX_PT3 + 1);
  c.take(B.sat, MAX_T5 + 1);
  c.take(B.sap, MAX_PLS + 1);
  c.take(B.tc_ev_off, 2);
  c.take(B.mask_off, MAX_MD);
  c.take(B.scan_state, (size_t)N_SCAN_SLOTS * STATIC_SCAN_CHUNKS);
  B.scan_chunks = STATIC_SCAN_CHUNKS;
  B.cap_mask = MASK_WORDS;
  c.take(B.mask, MASK_WORDS);
  return c.off;
}

constexpr size_t layout_bytes() {
  Sizer z;
  BufView B{};
  return carve_layout(z, B);
}
static_assert(layout_bytes() <= SCRATCH_BYTES, "the static scratch layout is larger than the scratch array");

__global__ void k_static_header(Hdr* H, Hdr v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *H = v;
}

const char* list_name(int t) {
  static const char* n[N_TOTALS] = {"hits", "MD", "LS", "T3", "T5", "pT3", "pT5", "MD-pT5 list", "MD-pT3 list",
                                    "MD-T5 list", "pT5 flags", "pT3 flags", "T5 flags", "pLS flags", "TC", "pT3 items"};
  return (t >= 0 && t < N_TOTALS) ? n[t] : "?";
}

// Device address of the scratch on `device`, looked up once (with that device current).
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[device] = p;
  }
  *out = g_scratch_dev[device];
  return cudaSuccess;
}

}  // namespace

namespace lst {
// Context set-up for the allocation-free entry point, run by lst_load_geometry with the
// context's device current: the scratch's device address (resolving it loads this file's
// module, and with it the array, on that device) and every kernel the chain launches, so
// that lst_run_event_static itself allocates nothing, not even on its first call.
cudaError_t static_scratch_prepare(int device) {
  if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
  void* p = nullptr;
  cudaError_t e = scratch_address(device, &p);
  if (e == cudaSuccess) {
    cudaFuncAttributes a;
    e = cudaFuncGetAttributes(&a, (const void*)k_static_header);
  }
  if (e == cudaSuccess) e = preload_kernels();
  return e;
}

// Test hook: the next call on `device` takes run tag e + 1 (LST_TEST_SCAN_EPOCH at context
// creation), so that tests can run across the point where the tags start again.
void static_scan_epoch_set(int device, uint32_t e) {
  if (device < 0 || device >= MAX_DEVICES) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_scan_epoch[device] = e & 0x3FFFFFFFu;
}
}  // namespace lst

extern "C" lst_status lst_run_event_static(lst_ctx* ctx, const lst_batch_dev* ev, lst_tc* tc_out, uint32_t tc_cap,
                                           uint32_t* n_tc, void* stream) {
  if (!ctx || !ev || !n_tc || (tc_cap && !tc_out)) return LST_ERR_INVALID_ARG;
  GeoView G;
  MethodConst C;
  Launch L;
  int dev = 0;
  bool have_map = false;
  if (!ctx_views(ctx, &G, &C, &L, &dev, &have_map)) return LST_ERR_INVALID_ARG;
  if (!have_map) {
    ctx_set_error(ctx, "lst_build_connection_map has not run");
    return LST_ERR_NO_MAP;
  }
  if (ev->n_events != 1 || !ev->hit_off || !ev->pls_off || (ev->n_hits && (!ev->x || !ev->y || !ev->z || !ev->det)) ||
      (ev->n_pls && !ev->pls)) {
    ctx_set_error(ctx, "lst_run_event_static takes exactly one event with device input pointers");
    return LST_ERR_INVALID_ARG;
  }
  if (ev->n_hits > MAX_HITS || ev->n_pls > MAX_PLS || G.nm > MAX_MODULES) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "event exceeds the static scratch: %u hits (max %u), %u pLS (max %u), %u modules (max %u)",
             ev->n_hits, MAX_HITS, ev->n_pls, MAX_PLS, G.nm, MAX_MODULES);
    ctx_set_error(ctx, msg);
    return LST_ERR_BUDGET;
  }
  if (dev < 0 || dev >= MAX_DEVICES) return LST_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) {
    ctx_set_error(ctx, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return LST_ERR_CUDA;
  }
  void* base = nullptr;
  // prepared by lst_load_geometry; looked up here only if that set-up could not run
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    ctx_set_error(ctx, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return LST_ERR_CUDA;
  }
  BufView B{};
  Placer place{(char*)base};
  carve_layout(place, B);
  B.cap_tc = tc_cap;
  B.tc = tc_out;
  cudaStream_t s = (cudaStream_t)stream;
  Hdr h{};
  h.x = ev->x; h.y = ev->y; h.z = ev->z; h.det = ev->det; h.hit_off = ev->hit_off;
  h.pls = (const PlsIn*)ev->pls; h.pls_off = ev->pls_off;
  h.n_ev = 1; h.n_hits = ev->n_hits; h.n_pls = ev->n_pls;
  bool clear_states = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scan_epoch[dev] == 0x3FFFFFFFu) {  // the tags would repeat: start again from clear states
      g_scan_epoch[dev] = 0;
      clear_states = true;
    }
    h.scan_epoch = ++g_scan_epoch[dev];
  }
  if (clear_states) {
    e = cudaMemsetAsync(B.scan_state, 0, (size_t)N_SCAN_SLOTS * STATIC_SCAN_CHUNKS * sizeof(*B.scan_state), s);
    if (e != cudaSuccess) {
      ctx_set_error(ctx, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
      return LST_ERR_CUDA;
    }
  }
  // the header (and with it every total and the error word) starts from zero on each call
  k_static_header<<<1, 32, 0, s>>>(B.hdr, h);
  const int launched = enqueue_pipeline(C, G, B, L, s, nullptr, nullptr);
  Hdr out;
  e = cudaGetLastError();
  if (e == cudaSuccess && launched <= 0) {
    ctx_set_error(ctx, "lst_run_event_static: the chain was not enqueued");
    return LST_ERR_CUDA;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&out, B.hdr, sizeof(Hdr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ctx_set_error(ctx, std::string("lst_run_event_static: ") + cudaGetErrorString(e));
    return LST_ERR_CUDA;
  }
  if (out.err & ERR_BAD_INPUT) {
    ctx_set_error(ctx, "bad input: module id out of range, non-finite value or invalid pLS");
    return LST_ERR_BAD_INPUT;
  }
  if (out.err & ERR_WAIT) {
    ctx_set_error(ctx, "a bounded device-side wait ran out");
    return LST_ERR_TIMEOUT;
  }
  const uint32_t ovf = out.err >> ERR_OVERFLOW_SHIFT;
  if (ovf & (1u << T_TC)) {
    *n_tc = out.tot[T_TC];
    ctx_set_error(ctx, "track-candidate buffer too small");
    return LST_ERR_BUFFER_TOO_SMALL;
  }
  if (ovf) {
    int t = 0;
    while (!(ovf & (1u << t))) t++;
    char msg[160];
    snprintf(msg, sizeof msg, "the %s list (%u entries) exceeds the static scratch of lst_run_event_static",
             list_name(t), out.tot[t]);
    ctx_set_error(ctx, msg);
    return LST_ERR_BUDGET;
  }
  *n_tc = out.tot[T_TC];
  return LST_OK;
}
