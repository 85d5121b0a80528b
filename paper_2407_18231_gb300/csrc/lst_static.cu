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

// The scratch.  In host code `g_scratch` is only a stand-in symbol: its device address
// comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_dev[MAX_DEVICES] = {};

struct Carver {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

// Lays every list of one event out in the scratch; returns the bytes used.
size_t carve(char* base, BufView& B) {
  Carver c{base, 0};
  B.hdr = c.take<Hdr>(1);
  B.cap_ev = 1; B.cap_hits = MAX_HITS; B.cap_md = MAX_MD; B.cap_ls = MAX_LS; B.cap_t3 = MAX_T3;
  B.cap_t5 = MAX_T5; B.cap_pls = MAX_PLS; B.cap_pt3 = MAX_PT3; B.cap_pt5 = MAX_PT5;
  B.sen_cnt = c.take<uint32_t>(2 * MAX_MODULES + 1);
  B.sen_off = c.take<uint32_t>(2 * MAX_MODULES + 1);
  B.hit_tmp = c.take<uint32_t>(MAX_HITS);
  B.hit_ev = c.take<uint32_t>(MAX_HITS);
  B.hit_idx = c.take<uint32_t>(MAX_HITS);
  B.hit4 = c.take<float4>(MAX_HITS);
  B.hit_sen = c.take<uint32_t>(MAX_HITS);
  B.md_hcnt = c.take<uint32_t>(MAX_HITS);
  B.md_hoff = c.take<uint32_t>(MAX_HITS + 1);
  B.md_hmask = c.take<uint32_t>(MAX_HITS);
  B.md_off = c.take<uint32_t>(MAX_MODULES + 1);
  B.md_box = c.take<float4>(2 * (size_t)MAX_MODULES);
  B.md_unit = c.take<uint32_t>(MAX_MD);
  B.md_lo_idx = c.take<uint32_t>(MAX_MD);
  B.md_up_idx = c.take<uint32_t>(MAX_MD);
  B.md_pt = c.take<float4>(2 * MAX_MD);
  B.md_up4 = c.take<float4>(MAX_MD);
  B.md_dir4 = c.take<float4>(MAX_MD);
  B.ls_cnt = c.take<uint32_t>(MAX_MD);
  B.ls_off = c.take<uint32_t>(MAX_MD + 1);
  B.ls_in = c.take<uint32_t>(MAX_LS);
  B.ls_out = c.take<uint32_t>(MAX_LS);
  B.t3_lcnt = c.take<uint32_t>(MAX_LS);
  B.t3_mask = c.take<uint32_t>(MAX_LS);
  B.t3_loff = c.take<uint32_t>(MAX_LS + 1);
  B.t3_off = c.take<uint32_t>(MAX_MD + 1);
  B.t3_a = c.take<uint32_t>(MAX_T3);
  B.t3_b = c.take<uint32_t>(MAX_T3);
  B.t3_c = c.take<uint32_t>(MAX_T3);
  B.t3_md4 = c.take<uint4>(MAX_T3);
  B.t5_tcnt = c.take<uint32_t>(MAX_T3);
  B.t5_mask = c.take<uint32_t>(MAX_T3);
  B.t5_toff = c.take<uint32_t>(MAX_T3 + 1);
  B.t5_off = c.take<uint32_t>(MAX_MD + 1);
  B.t5_m0 = c.take<uint32_t>(MAX_T5);
  B.t5_m1 = c.take<uint32_t>(MAX_T5);
  B.t5_m2 = c.take<uint32_t>(MAX_T5);
  B.t5_m3 = c.take<uint32_t>(MAX_T5);
  B.t5_m4 = c.take<uint32_t>(MAX_T5);
  B.t5_score = c.take<float>(MAX_T5);
  B.t5_kfull = c.take<float>(MAX_T5);
  B.t5_md8 = c.take<uint4>(2 * MAX_T5);
  B.pls_ev = c.take<uint32_t>(MAX_PLS);
  B.pls_ncand = c.take<uint32_t>(MAX_PLS);
  B.pls_cand = c.take<uint32_t>((size_t)MAX_PLS * MAX_CAND);
  B.pls_mdpass = c.take<uint32_t>((size_t)MAX_PLS * PLS_MD_CAP);
  B.pls_nmdpass = c.take<uint32_t>(MAX_PLS);
  B.pls_h0 = c.take<float4>(MAX_PLS);
  B.pls_h1 = c.take<float4>(MAX_PLS);
  B.pls_pt = c.take<float>(MAX_PLS);
  B.pt3_icnt = c.take<uint32_t>(MAX_PLS);
  B.pt3_ioff = c.take<uint32_t>(MAX_PLS + 1);
  B.pt3_item_p = c.take<uint32_t>((size_t)MAX_PLS * PLS_ITEMS);
  B.pt3_xcnt = c.take<uint32_t>((size_t)MAX_PLS * PLS_ITEMS);
  B.pt3_xoff = c.take<uint32_t>((size_t)MAX_PLS * PLS_ITEMS + 1);
  B.pt3_xmask = c.take<uint32_t>((size_t)MAX_PLS * PLS_ITEMS);
  B.pt3_off = c.take<uint32_t>(MAX_PLS + 1);
  B.pt3_pls = c.take<uint32_t>(MAX_PT3);
  B.pt3_obj = c.take<uint32_t>(MAX_PT3);
  B.pt3_score = c.take<float>(MAX_PT3);
  B.pt5_xcnt = c.take<uint32_t>(MAX_PT3);
  B.pt5_xoff = c.take<uint32_t>(MAX_PT3 + 1);
  B.pt5_xmask = c.take<uint32_t>(MAX_PT3);
  B.pt5_off = c.take<uint32_t>(MAX_PLS + 1);
  B.pt5_pls = c.take<uint32_t>(MAX_PT5);
  B.pt5_obj = c.take<uint32_t>(MAX_PT5);
  B.pt5_score = c.take<float>(MAX_PT5);
  B.c5_cnt = c.take<uint32_t>(MAX_MD + 1);
  B.c5_off = c.take<uint32_t>(MAX_MD + 1);
  B.c5_list = c.take<uint32_t>((size_t)5 * MAX_PT5);
  B.c3_cnt = c.take<uint32_t>(MAX_MD + 1);
  B.c3_off = c.take<uint32_t>(MAX_MD + 1);
  B.c3_list = c.take<uint32_t>((size_t)3 * MAX_PT3);
  B.ct_cnt = c.take<uint32_t>(MAX_MD + 1);
  B.ct_off = c.take<uint32_t>(MAX_MD + 1);
  B.ct_list = c.take<uint32_t>((size_t)5 * MAX_T5);
  B.alive5 = c.take<uint32_t>(MAX_PT5);
  B.alive3 = c.take<uint32_t>(MAX_PT3);
  B.alivet = c.take<uint32_t>(MAX_T5);
  B.plstc = c.take<uint32_t>(MAX_PLS);
  B.cross3 = c.take<uint32_t>(MAX_PT3);
  B.crosst = c.take<uint32_t>(MAX_T5);
  B.sa5 = c.take<uint32_t>(MAX_PT5 + 1);
  B.sa3 = c.take<uint32_t>(MAX_PT3 + 1);
  B.sat = c.take<uint32_t>(MAX_T5 + 1);
  B.sap = c.take<uint32_t>(MAX_PLS + 1);
  B.tc_ev_off = c.take<uint32_t>(2);
  B.scan_part = c.take<uint32_t>(4 * 1024);  // partials of up to four scans per launch
  B.scan_part2 = c.take<uint32_t>(1024);
  B.mask_off = c.take<uint32_t>(MAX_MD);
  B.cap_mask = MASK_WORDS;
  B.mask = c.take<uint32_t>(MASK_WORDS);
  return c.off;
}

__global__ void k_static_header(Hdr* H, Hdr v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *H = v;
}

const char* list_name(int t) {
  static const char* n[N_TOTALS] = {"hits", "MD", "LS", "T3", "T5", "pT3", "pT5", "MD-pT5 list", "MD-pT3 list",
                                    "MD-T5 list", "pT5 flags", "pT3 flags", "T5 flags", "pLS flags", "TC", "pT3 items"};
  return (t >= 0 && t < N_TOTALS) ? n[t] : "?";
}

}  // namespace

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
  {
    // once per device, with that device current: the device address of the scratch
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) {
        ctx_set_error(ctx, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return LST_ERR_CUDA;
      }
      BufView probe;
      if (carve((char*)p, probe) > SCRATCH_BYTES) {
        ctx_set_error(ctx, "static scratch layout larger than the scratch array");
        return LST_ERR_BUDGET;
      }
      g_scratch_dev[dev] = p;
    }
    base = g_scratch_dev[dev];
  }
  BufView B;
  carve((char*)base, B);
  B.cap_tc = tc_cap;
  B.tc = tc_out;
  cudaStream_t s = (cudaStream_t)stream;
  Hdr h{};
  h.x = ev->x; h.y = ev->y; h.z = ev->z; h.det = ev->det; h.hit_off = ev->hit_off;
  h.pls = (const PlsIn*)ev->pls; h.pls_off = ev->pls_off;
  h.n_ev = 1; h.n_hits = ev->n_hits; h.n_pls = ev->n_pls;
  // the header (and with it every total and the error word) starts from zero on each call
  k_static_header<<<1, 32, 0, s>>>(B.hdr, h);
  enqueue_pipeline(C, G, B, L, s, nullptr, nullptr);
  Hdr out;
  e = cudaGetLastError();
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
