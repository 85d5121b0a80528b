// Host runtime of liblst: geometry tables, connection map, device buffers, CUDA-graph
// replay, results, the C ABI and the continuous-batching serving loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <mutex>
#include <condition_variable>
#include <atomic>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lst.h"
#include "lst_device.cuh"

namespace lst {
int enqueue_pipeline(const MethodConst& C, const GeoView& G, const BufView& B, const Launch& L, cudaStream_t s,
                     MarkFn mark, void* arg, const SideBranch* side = nullptr);
cudaError_t static_scratch_prepare(int device);  // lst_static.cu
void static_scan_epoch_set(int device, uint32_t e);  // lst_static.cu
cudaError_t configure_kernels();
}

using namespace lst;

namespace {

// ------------------------------------------------------------------ method constants
// pT = KB * R with KB = 0.0029979 * 3.8; Rmin is the radius of a 0.8 GeV track (Sec. 1).
const double KB_D = 0.0029979245800 * 3.8;
const double RMIN_D = 0.8 / KB_D;

MethodConst method_constants() {
  MethodConst c;
  c.KB = (float)KB_D;
  c.Z0MAX = 15.0f;
  c.E0 = 0.03f;
  c.KARC = (float)(2.0 / (24.0 * RMIN_D * RMIN_D));
  c.K3 = (float)(2.0 * RMIN_D * 0.95);
  c.KMAX = (float)(1.0 / (RMIN_D * 0.95));
  c.KAPPA = 0.05f;
  c.KAPPA0 = 1.0e-4f;
  c.KPT5 = 0.15f;
  c.W0 = 0.02f;
  c.PI = 3.14159265f;
  c.HINV = (float)(1.0 / (2.0 * RMIN_D));
  c.EDIR = 0.013f;
  return c;
}

// ------------------------------------------------------------------ helpers
struct CudaError {
  cudaError_t e;
  const char* what;
};
#define CK(x)                                         \
  do {                                                \
    cudaError_t _e = (x);                             \
    if (_e != cudaSuccess) throw CudaError{_e, #x};   \
  } while (0)

struct StatusError {
  lst_status s;
  std::string msg;
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int surface_of(const lst_module_desc& m) {
  if (m.subdet == 0) return (m.layer >= 1 && m.layer <= 6) ? m.layer - 1 : -1;
  if (m.subdet == 1 && m.layer >= 1 && m.layer <= 5) {
    if (m.side < 0) return 6 + m.layer - 1;
    if (m.side > 0) return 11 + m.layer - 1;
  }
  return -1;
}

// ------------------------------------------------------------------ device buffer
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t b, uint64_t& total) {
    if (b <= bytes) return;
    if (p) {
      cudaFree(p);
      total -= bytes;
    }
    p = nullptr;
    bytes = 0;
    CK(cudaMalloc(&p, b));
    bytes = b;
    total += b;
  }
};

// ------------------------------------------------------------------ geometry
struct Geometry {
  std::vector<lst_module_desc> mods;
  uint32_t nm = 0;
  std::vector<float4> modc;  // zeta, rho, delta, T
  std::vector<float> rnext;
  std::vector<uint8_t> subdet;
  std::vector<int> surface;
  float zb_half = 0.0f;
  int32_t surf_first[NSURF];
  uint32_t surf_nrows[NSURF];
  uint32_t surf_row_base[NSURF];
  std::vector<uint32_t> row_nphi, row_mod_base, row_mods;
  std::vector<uint8_t> row_fast;
  std::vector<float> row_phi0;
  std::vector<uint32_t> conn_off, conn;
  std::vector<float> conn_dpsi;  // per map edge: pseudo-angle half-width of the LS bending window
  bool have_map = false;
  // learned T5 selection (passed to the T5 kernels by value); sel_version counts changes so
  // that every pipeline re-captures its graph after one
  bool has_t5_mlp = false;
  T5Mlp t5_mlp{};
  uint32_t sel_version = 0;
  // device copies
  DevBuf d_modc, d_rnext, d_subdet, d_mod_e, d_mod_g, d_row_nphi, d_row_base, d_row_mods, d_conn_off, d_conn,
      d_row_fast, d_row_phi0, d_conn_dpsi;
  uint64_t dev_bytes = 0;

  ~Geometry() {
    DevBuf* all[] = {&d_modc, &d_rnext, &d_subdet, &d_mod_e, &d_mod_g, &d_row_nphi, &d_row_base,
                     &d_row_mods, &d_conn_off, &d_conn, &d_row_fast, &d_row_phi0, &d_conn_dpsi};
    for (DevBuf* b : all) b->release();
  }

  void load(const lst_module_desc* m, uint32_t n) {
    mods.assign(m, m + n);
    nm = n;
    modc.resize(n);
    rnext.resize(n);
    subdet.resize(n);
    surface.resize(n);
    for (int s = 0; s < NSURF; s++) {
      surf_first[s] = -1;
      surf_nrows[s] = 0;
    }
    float rlay[6] = {0, 0, 0, 0, 0, 0};
    bool have[6] = {false, false, false, false, false, false};
    zb_half = 0.0f;
    for (uint32_t i = 0; i < n; i++) {
      const lst_module_desc& d = mods[i];
      const int s = surface_of(d);
      if (s < 0 || d.nphi == 0 || d.iphi >= d.nphi || !std::isfinite(d.surf) || !std::isfinite(d.gap) ||
          !std::isfinite(d.emin) || !std::isfinite(d.emax) || !(d.emax > d.emin) || !(std::fabs(d.tilt) < 1.5f) ||
          (d.subdet != 0 && d.tilt != 0.0f))
        throw StatusError{LST_ERR_BAD_INPUT, "module " + std::to_string(i) + " is malformed"};
      surface[i] = s;
      subdet[i] = d.subdet;
      // bending slope at the module's largest radius (the upper sensor of a tilted module
      // included), tolerances of its hits: a tilted PS module's coarse coordinate runs
      // along its surface, so 3 x 0.5 mm projects onto both z and r; an endcap 2S module
      // gives r to half a 5 cm strip
      double rmax;
      if (d.subdet == 0) {
        const double t = (double)d.tilt;
        rmax = (double)d.surf + 0.5 * ((double)d.emax - (double)d.emin) * std::fabs(std::tan(t)) +
               (double)d.gap * std::cos(t);
      } else {
        rmax = (double)d.emax;
      }
      const double sq = rmax / (2.0 * RMIN_D);
      const float T = (float)(sq < 1.0 ? sq / std::sqrt(1.0 - sq * sq) : 1.0e30);
      float zeta, rho;
      if (d.subdet == 0) {
        if (d.tilt != 0.0f) {
          zeta = (float)(0.15 * std::fabs(std::cos((double)d.tilt)));
          rho = (float)(0.15 * std::fabs(std::sin((double)d.tilt)));
        } else {
          zeta = d.stype == 0 ? 0.15f : 1.30f;
          rho = 0.0f;
        }
      } else {
        zeta = 0.0f;
        rho = d.stype == 0 ? 0.15f : 2.55f;
      }
      const float delta = 0.01f + rho;
      modc[i] = make_float4(zeta, rho, delta, T);
      if (surf_first[s] < 0) surf_first[s] = (int32_t)i;
      surf_nrows[s] = std::max<uint32_t>(surf_nrows[s], d.ieta + 1u);
      if (d.subdet == 0) {
        rlay[d.layer - 1] = d.surf;
        have[d.layer - 1] = true;
        zb_half = std::max(zb_half, std::fabs(d.emin));
        zb_half = std::max(zb_half, std::fabs(d.emax));
      }
    }
    for (uint32_t i = 0; i < n; i++) {
      const lst_module_desc& d = mods[i];
      rnext[i] = 1.0e30f;
      if (d.subdet == 0 && d.layer < 6 && have[d.layer]) rnext[i] = rlay[d.layer];
    }
    // rows (z bins / rings) of each surface, indexed by iphi
    uint32_t nrows = 0;
    for (int s = 0; s < NSURF; s++) {
      surf_row_base[s] = nrows;
      nrows += surf_nrows[s];
    }
    row_nphi.assign(nrows, 0);
    row_mod_base.assign(nrows, 0);
    for (uint32_t i = 0; i < n; i++) {
      const uint32_t r = surf_row_base[surface[i]] + mods[i].ieta;
      if (row_nphi[r] != 0 && row_nphi[r] != mods[i].nphi)
        throw StatusError{LST_ERR_BAD_INPUT, "row with two sector counts"};
      row_nphi[r] = mods[i].nphi;
    }
    uint32_t tot = 0;
    for (uint32_t r = 0; r < nrows; r++) {
      row_mod_base[r] = tot;
      tot += row_nphi[r];
    }
    row_mods.assign(std::max<uint32_t>(tot, 1), NONE);
    for (uint32_t i = 0; i < n; i++) {
      const uint32_t r = surf_row_base[surface[i]] + mods[i].ieta;
      uint32_t& slot = row_mods[row_mod_base[r] + mods[i].iphi];
      if (slot != NONE) throw StatusError{LST_ERR_BAD_INPUT, "two modules share a row and sector"};
      slot = i;
    }
    // rows whose sectors partition the circle
    row_fast.assign(nrows, 0);
    row_phi0.assign(nrows, 0.0f);
    for (uint32_t r = 0; r < nrows; r++) {
      const uint32_t n = row_nphi[r];
      if (n < 3) continue;
      bool ok = true;
      for (uint32_t k = 0; k < n && ok; k++) {
        const uint32_t a = row_mods[row_mod_base[r] + k], b = row_mods[row_mod_base[r] + (k + 1) % n];
        if (a == NONE || b == NONE) { ok = false; break; }
        const lst_module_desc &ma = mods[a], &mb = mods[b];
        ok = ma.e1x == mb.e0x && ma.e1y == mb.e0y &&
             (double)ma.e0x * ma.e1y - (double)ma.e0y * ma.e1x > 0.0;
      }
      if (!ok) continue;
      row_fast[r] = 1;
      const lst_module_desc& m0 = mods[row_mods[row_mod_base[r]]];
      row_phi0[r] = (float)std::atan2((double)m0.e0y, (double)m0.e0x);
    }
  }

  // ---- connection map: conservative bound of the LS selection over module pairs ----
  struct Box {
    double r0, r1, z0, z1;  // anchor ranges
    double phic, phih;      // wedge centre and half width
  };
  Box box_of(uint32_t i) const {
    const lst_module_desc& d = mods[i];
    Box b;
    if (d.subdet == 0 && d.tilt != 0.0f) {  // a tilted section spans surf +- half its z length x |tan(tilt)|
      const double h = 0.5 * ((double)d.emax - (double)d.emin) * std::fabs(std::tan((double)d.tilt));
      b.r0 = d.surf - h - 0.5; b.r1 = d.surf + h + 0.5;
      b.z0 = d.emin - 0.5; b.z1 = d.emax + 0.5;
    } else if (d.subdet == 0) {
      b.r0 = d.surf - 0.01; b.r1 = d.surf + 0.01;
      b.z0 = d.emin - 0.5; b.z1 = d.emax + 0.5;
    } else {
      b.z0 = d.surf - 0.01; b.z1 = d.surf + 0.01;
      b.r0 = d.emin - 0.5; b.r1 = d.emax + 0.5;
    }
    const double a0 = std::atan2((double)d.e0y, (double)d.e0x);
    double w = std::atan2((double)d.e1y, (double)d.e1x) - a0;
    while (w <= 0) w += 2 * M_PI;
    b.phih = 0.5 * w;
    b.phic = a0 + 0.5 * w;
    return b;
  }

  // Largest azimuth difference |d| = |phi_b - phi_a| of an anchor pair (a in A, b in B)
  // that can pass the LS bending cut.  With U = r_a r_b sin(d), W = r_a (r_b cos(d) - r_a +
  // rs) and E = (e0 + rs (|sin(d)| + 0.05)) r_a, the cut |U| <= W T_B + E, W > 0 gives
  // cos(d) > 0 and |sin(d)| <= (1 - (r_a - rs) / r_b) T_B + e_max / r_b, e_max = e0 + 1.05 rs,
  // which is largest at the smallest r_a of A's box and at an end of B's radius range; plus
  // 3 mrad for the rounding of the binary32 test.
  double bend_dphi(uint32_t A, uint32_t Bm, const Box& a, const Box& b) const {
    const double rs = (double)modc[A].y + (double)modc[Bm].y;
    const double emax = 0.03 + 1.05 * rs;
    const double T = (double)modc[Bm].w;
    auto bound = [&](double rb) { return (1.0 - (a.r0 - rs) / rb) * T + emax / rb; };
    const double S = std::max(bound(b.r0), bound(b.r1));
    return (S >= 1.0 ? 0.5 * M_PI : std::asin(S)) + 3.0e-3;
  }

  // Can some anchor in A and some anchor in B pass the LS bending and r-z cuts?
  bool reachable(uint32_t A, uint32_t Bm, const Box& a, const Box& b) const {
    const double dphi = bend_dphi(A, Bm, a, b);
    double d = std::fmod(a.phic - b.phic, 2 * M_PI);
    if (d > M_PI) d -= 2 * M_PI;
    if (d < -M_PI) d += 2 * M_PI;
    if (std::fabs(d) > a.phih + b.phih + dphi) return false;
    // r-z cut: za rb - ra zb is multilinear, so its range over the box is spanned by the
    // 16 corners; the tolerance is bounded by its largest value over the box
    double lo = 1e300, hi = -1e300;
    for (int c = 0; c < 16; c++) {
      const double za = (c & 1) ? a.z1 : a.z0, ra = (c & 2) ? a.r1 : a.r0;
      const double zb = (c & 4) ? b.z1 : b.z0, rb = (c & 8) ? b.r1 : b.r0;
      const double f = za * rb - ra * zb;
      lo = std::min(lo, f);
      hi = std::max(hi, f);
    }
    const double fmin = (lo <= 0 && hi >= 0) ? 0.0 : std::min(std::fabs(lo), std::fabs(hi));
    const double drmax = std::max(std::fabs(b.r1 - a.r0), std::fabs(b.r0 - a.r1));
    const double zbm = std::max(std::fabs(b.z0), std::fabs(b.z1));
    const double zam = std::max(std::fabs(a.z0), std::fabs(a.z1));
    const double dzm = std::max(std::fabs(b.z1 - a.z0), std::fabs(b.z0 - a.z1));
    const double karc = 2.0 / (24.0 * RMIN_D * RMIN_D);
    const double tol = 15.0 * drmax + modc[A].x * b.r1 + modc[Bm].x * a.r1 + modc[A].y * zbm + modc[Bm].y * zam +
                       karc * dzm * a.r1 * b.r1 * (a.r1 + b.r1);
    return fmin <= tol * 1.01 + 0.01;
  }

  void build_map() {
    std::vector<Box> boxes(nm);
    for (uint32_t i = 0; i < nm; i++) boxes[i] = box_of(i);
    std::vector<std::vector<uint32_t>> by_surface(NSURF);
    for (uint32_t i = 0; i < nm; i++) by_surface[surface[i]].push_back(i);
    conn_off.assign(nm + 1, 0);
    conn.clear();
    conn_dpsi.clear();
    for (uint32_t A = 0; A < nm; A++) {
      conn_off[A] = (uint32_t)conn.size();
      const int s = surface[A];
      int next[3], k = 0;
      if (s < 6) {  // barrel layer: next layer, or out through the first disk of either side
        if (s < 5) next[k++] = s + 1;
        next[k++] = 6;
        next[k++] = 11;
      } else if ((s < 11 && s < 10) || (s >= 11 && s < 15)) {
        next[k++] = s + 1;  // next disk on the same side
      }
      std::vector<uint32_t> nbr;
      for (int t = 0; t < k; t++)
        for (uint32_t Bm : by_surface[next[t]])
          if (reachable(A, Bm, boxes[A], boxes[Bm])) nbr.push_back(Bm);
      std::sort(nbr.begin(), nbr.end());
      for (uint32_t Bm : nbr) {
        conn.push_back(Bm);
        // the azimuth bound as a pseudo-angle half-width (|d psi| <= |d phi|), rounded up
        conn_dpsi.push_back((float)(bend_dphi(A, Bm, boxes[A], boxes[Bm]) * (1.0 + 1e-6) + 1e-4));
      }
    }
    conn_off[nm] = (uint32_t)conn.size();
    have_map = true;
  }

  template <typename T>
  void upload(DevBuf& b, const std::vector<T>& v) {
    b.ensure(std::max<size_t>(v.size(), 1) * sizeof(T), dev_bytes);
    if (!v.empty()) CK(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  }

  void upload_tables() {
    std::vector<float4> e(nm), g(nm);
    for (uint32_t i = 0; i < nm; i++) {
      e[i] = make_float4(mods[i].e0x, mods[i].e0y, mods[i].e1x, mods[i].e1y);
      g[i] = make_float4(mods[i].surf, mods[i].gap, mods[i].emin, mods[i].emax);
    }
    upload(d_modc, modc);
    upload(d_rnext, rnext);
    upload(d_subdet, subdet);
    upload(d_mod_e, e);
    upload(d_mod_g, g);
    upload(d_row_nphi, row_nphi);
    upload(d_row_base, row_mod_base);
    upload(d_row_mods, row_mods);
    upload(d_row_fast, row_fast);
    upload(d_row_phi0, row_phi0);
  }

  void upload_map() {
    upload(d_conn_off, conn_off);
    upload(d_conn, conn);
    upload(d_conn_dpsi, conn_dpsi);
  }

  GeoView view() const {
    GeoView v;
    v.nm = nm;
    v.zb_half = zb_half;
    v.modc = (const float4*)d_modc.p;
    v.rnext = (const float*)d_rnext.p;
    v.subdet = (const uint8_t*)d_subdet.p;
    v.conn_off = (const uint32_t*)d_conn_off.p;
    v.conn = (const uint32_t*)d_conn.p;
    v.conn_dpsi = (const float*)d_conn_dpsi.p;
    v.mod_e = (const float4*)d_mod_e.p;
    v.mod_g = (const float4*)d_mod_g.p;
    for (int s = 0; s < NSURF; s++) {
      v.surf_first[s] = surf_first[s];
      v.surf_nrows[s] = surf_nrows[s];
      v.surf_row_base[s] = surf_row_base[s];
    }
    v.row_nphi = (const uint32_t*)d_row_nphi.p;
    v.row_mod_base = (const uint32_t*)d_row_base.p;
    v.row_mods = (const uint32_t*)d_row_mods.p;
    v.row_fast = (const uint8_t*)d_row_fast.p;
    v.row_phi0 = (const float*)d_row_phi0.p;
    return v;
  }
};

// ------------------------------------------------------------------ host copy workers
// A fixed set of helper threads for the host-side copies of a batch (packing the inputs
// into pinned staging, unpacking the candidates): run(n, fn) calls fn(0..n-1) on the helpers
// and the caller and returns when all calls are done.  One per pipeline, so batch slots
// served concurrently never share it.
class Workers {
 public:
  explicit Workers(unsigned n_helpers) {
    for (unsigned i = 0; i < n_helpers; i++) th_.emplace_back([this] { loop(); });
  }
  ~Workers() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  void run(uint32_t n, const std::function<void(uint32_t)>& fn) {
    if (n == 0) return;
    uint64_t g;
    {
      std::lock_guard<std::mutex> lk(m_);
      fn_ = &fn;
      n_ = n;
      next_ = 0;
      left_ = n;
      g = ++gen_;
    }
    cv_.notify_all();
    work(g, &fn);
    std::unique_lock<std::mutex> lk(m_);
    done_cv_.wait(lk, [this] { return left_ == 0; });
  }

 private:
  // tasks are claimed under the lock and only for the job of generation g, so a helper
  // that wakes after its job has ended never runs a later job's task with a stale fn
  bool claim(uint64_t g, uint32_t& i) {
    std::lock_guard<std::mutex> lk(m_);
    if (gen_ != g || next_ >= n_) return false;
    i = next_++;
    return true;
  }
  void work(uint64_t g, const std::function<void(uint32_t)>* fn) {
    uint32_t i;
    while (claim(g, i)) {
      (*fn)(i);
      std::lock_guard<std::mutex> lk(m_);
      if (--left_ == 0) done_cv_.notify_all();
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(uint32_t)>* fn;
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        fn = fn_;
      }
      work(seen, fn);
    }
  }
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(uint32_t)>* fn_ = nullptr;
  uint32_t n_ = 0, next_ = 0, left_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// ------------------------------------------------------------------ results
struct Result {
  std::shared_ptr<const lst_tc[]> tc_buf;  // the batch's candidates
  size_t tc_off = 0, tc_n = 0;             // this event's slice
  bool has_objects = false;
  std::vector<lst_md_rec> md;
  std::vector<lst_ls_rec> ls;
  std::vector<lst_t3_rec> t3;
  std::vector<lst_t5_rec> t5;
  std::vector<lst_px_rec> pt3, pt5;
  std::vector<lst_pls_rec> pls;
};

// ------------------------------------------------------------------ capacities
struct Caps {
  uint32_t ev = 0, hits = 0, pls = 0, md = 0, ls = 0, t3 = 0, t5 = 0, pt3 = 0, pt5 = 0, tc = 0;
};

// ------------------------------------------------------------------ pipeline (one batch slot)
struct Pipeline {
  Geometry* geo = nullptr;
  MethodConst C;
  Launch L;
  cudaStream_t stream = nullptr;
  SideBranch side{nullptr, nullptr, nullptr, nullptr};  // second stream of the chain (not in profile mode)
  cudaEvent_t done = nullptr;
  Caps cap;
  uint64_t dev_bytes = 0;
  // learned object-per-hit ratios for sizing (grow only)
  double r_md = 0.6, r_ls = 1.5, r_t3 = 1.0, r_t5 = 0.3, r_pt3 = 6.0, r_pt5 = 6.0;
  // buffers
  DevBuf hdr, in_x, in_y, in_z, in_det, in_hoff, in_pls, in_poff;
  DevBuf sen_cnt, sen_off, hit_tmp, hit_psi, hit_ev, hit_idx, hit_sen, hit4;
  DevBuf md_hcnt, md_hoff, md_hmask, md_box, md_off, md_unit, md_lo_idx, md_up_idx, md_pt, md_up4, md_dir4, md_psi;
  DevBuf ls_cnt, ls_off, ls_in, ls_out;
  DevBuf t3_lcnt, t3_loff, t3_off, t3_a, t3_b, t3_c, t3_mask, t3_md4;
  DevBuf t5_tcnt, t5_toff, t5_off, t5_m[5], t5_score, t5_kfull, t5_mask, t5_md8;
  DevBuf pls_ev, pls_ncand, pls_cand, pls_h0, pls_h1, pls_pt, pls_mdpass, pls_nmdpass;
  DevBuf pt3_icnt, pt3_ioff, pt3_item_p, pt3_xcnt, pt3_xoff, pt3_xmask, pt3_off, pt3_pls, pt3_obj, pt3_score;
  DevBuf pt5_xcnt, pt5_xoff, pt5_xmask, pt5_off, pt5_pls, pt5_obj, pt5_score;
  DevBuf c5_cnt, c5_off, c5_list, c3_cnt, c3_off, c3_list, ct_cnt, ct_off, ct_list;
  DevBuf alive5, alive3, alivet, plstc, cross3, crosst, sa5, sa3, sat, sap;
  DevBuf tc_ev_off, tc, mask, mask_off, scan_state;
  uint32_t scan_chunks = 1;  // chunk states per scan slot of the large single-pass scans
  uint32_t epoch = 0;        // runs launched (tags the chunk states; 30 bits)
  uint32_t cap_mask = 0;
  uint64_t byte_cap = 0;  // 0: none; otherwise learn_mask keeps dev_bytes within it
  bool auto_list_cap = true;  // the LS list cap is the library's choice (learn may raise it)
  // test hook for the bounded device waits: the next stall_scan_runs launches start every
  // single-pass scan's tickets at 1, so no block takes chunk 0 and the blocks of the later
  // chunks wait for a state that nothing writes until their polls run out
  // (LST_TEST_STALL_SCAN at context creation)
  uint32_t stall_scan_runs = 0;
  // test hook for the LS partner-list arena: when set, the arena holds this many words and
  // never grows, so that most anchors find it exhausted and are joined again by the fill
  // pass (LST_TEST_MASK_WORDS at context creation)
  uint32_t test_mask_words = 0;
  // host staging (pinned)
  Hdr* h_hdr = nullptr;        // header to upload
  Hdr* h_hdr_out = nullptr;    // header read back
  void* h_stage = nullptr;
  size_t h_stage_bytes = 0;
  lst_tc* h_tc = nullptr;  // pinned landing area of the candidates
  size_t h_tc_cap = 0;
  std::unique_ptr<Workers> workers;  // host copy helpers (created on first use)
  Workers& copiers() {
    if (!workers) {
      const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
      workers.reset(new Workers(std::min(hw, 16u) - 1));
    }
    return *workers;
  }
  // graph
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  uint32_t graph_sel_version = 0;  // the geometry's selection the graph was captured with
  int kernels = 0;
  // profile mode: one event after every kernel of an eager run
  bool profile = false;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<int> prof_name;
  cudaEvent_t prof_start = nullptr;
  // in-flight batch bookkeeping (serving / device path)
  uint32_t n_ev = 0, n_hits = 0, n_pls = 0;
  Hdr dev_inputs{};  // input pointers and sizes of the batch being run
  bool pending = false;

  ~Pipeline() { release(); }

  std::vector<DevBuf*> all_buffers() {
    std::vector<DevBuf*> v = {&hdr, &in_x, &in_y, &in_z, &in_det, &in_hoff, &in_pls, &in_poff, &sen_cnt, &sen_off,
                              &hit_tmp, &hit_psi, &hit_ev, &hit_idx, &hit_sen, &hit4, &md_hcnt, &md_hoff, &md_hmask, &md_box, &md_off, &md_unit, &md_lo_idx, &md_up_idx,
                              &md_pt, &md_up4, &md_dir4, &md_psi, &ls_cnt, &ls_off, &ls_in, &ls_out, &t3_lcnt, &t3_loff, &t3_off, &t3_mask, &t5_mask, &t3_md4, &t5_md8,
                              &t3_a, &t3_b, &t3_c, &t5_tcnt, &t5_toff, &t5_off, &t5_score, &t5_kfull, &pls_ev,
                              &pls_ncand, &pls_cand, &pls_h0, &pls_h1, &pls_pt, &pls_mdpass, &pls_nmdpass, &pt3_icnt, &pt3_ioff, &pt3_item_p, &pt3_xcnt, &pt3_xoff, &pt3_xmask, &pt3_off, &pt3_pls, &pt3_obj, &pt3_score,
                              &pt5_xcnt, &pt5_xoff, &pt5_xmask, &pt5_off, &pt5_pls, &pt5_obj, &pt5_score, &c5_cnt, &c5_off, &c5_list,
                              &c3_cnt, &c3_off, &c3_list, &ct_cnt, &ct_off, &ct_list, &alive5, &alive3, &alivet,
                              &plstc, &cross3, &crosst, &sa5, &sa3, &sat, &sap, &tc_ev_off, &tc,
                              &mask, &mask_off, &scan_state};
    for (auto& b : t5_m) v.push_back(&b);
    return v;
  }

  void release() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
    graph_valid = false;
    for (DevBuf* b : all_buffers()) b->release();
    dev_bytes = 0;
    if (h_hdr) cudaFreeHost(h_hdr);
    if (h_hdr_out) cudaFreeHost(h_hdr_out);
    workers.reset();
    if (h_tc) cudaFreeHost(h_tc);
    h_tc = nullptr;
    h_tc_cap = 0;
    if (h_stage) cudaFreeHost(h_stage);
    h_hdr = h_hdr_out = nullptr;
    h_stage = nullptr;
    h_stage_bytes = 0;
    for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
    prof_ev.clear();
    if (prof_start) cudaEventDestroy(prof_start);
    prof_start = nullptr;
    if (done) cudaEventDestroy(done);
    if (stream) cudaStreamDestroy(stream);
    done = nullptr;
    stream = nullptr;
    if (side.fork) cudaEventDestroy(side.fork);
    if (side.mds) cudaEventDestroy(side.mds);
    if (side.join) cudaEventDestroy(side.join);
    if (side.s) cudaStreamDestroy(side.s);
    side = SideBranch{nullptr, nullptr, nullptr, nullptr};
  }

  void set_tuning(const lst_config& cfg, int n_sm) {
    const uint32_t bps = cfg.blocks_per_sm ? cfg.blocks_per_sm : 4;
    L.block = cfg.block_size ? cfg.block_size : 256;
    // a multiple of 4: the LS kernel's per-warp shared-memory slices hold float4s
    L.ls_list_cap = cfg.ls_list_cap == 0 ? 512u
                                         : (cfg.ls_list_cap == 1 ? 0u : std::min(cfg.ls_list_cap, LS_LIST_MAX) & ~3u);
    auto_list_cap = cfg.ls_list_cap == 0;
    L.grid = (uint32_t)n_sm * bps;
    graph_valid = false;
  }

  void init(Geometry* g, const lst_config& cfg, int n_sm) {
    geo = g;
    C = method_constants();
    set_tuning(cfg, n_sm);
    CK(configure_kernels());
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&side.mds, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming));
    profile = cfg.profile != 0;
    if (profile) {
      CK(cudaEventCreate(&prof_start));
      prof_ev.resize(160);
      for (auto& e : prof_ev) CK(cudaEventCreate(&e));
    }
    CK(cudaMallocHost((void**)&h_hdr, sizeof(Hdr)));
    CK(cudaMallocHost((void**)&h_hdr_out, sizeof(Hdr)));
    hdr.ensure(sizeof(Hdr), dev_bytes);
  }

  template <typename T>
  void need(DevBuf& b, size_t n) {
    const size_t before = b.bytes;
    b.ensure(std::max<size_t>(n, 1) * sizeof(T), dev_bytes);
    if (b.bytes != before) graph_valid = false;
  }

  // Capacities c merged with the current ones (buffers never shrink).
  Caps merged(const Caps& c_in) const {
    Caps c = c_in;
    c.ev = std::max(c.ev, cap.ev);
    c.hits = std::max(c.hits, cap.hits);
    c.pls = std::max(c.pls, cap.pls);
    c.md = std::max(c.md, cap.md);
    c.ls = std::max(c.ls, cap.ls);
    c.t3 = std::max(c.t3, cap.t3);
    c.t5 = std::max(c.t5, cap.t5);
    c.pt3 = std::max(c.pt3, cap.pt3);
    c.pt5 = std::max(c.pt5, cap.pt5);
    c.tc = std::max(c.tc, cap.tc);
    return c;
  }

  // LS partner lists: about two words per hit suffice for PU200-like events; runs that
  // need more fall back to joining again and the next run gets the learned size
  uint32_t mask_words(const Caps& c) const {
    if (test_mask_words) return test_mask_words;
    return std::max<uint32_t>(cap_mask, (uint32_t)std::min<uint64_t>(4000000000ull, 4ull * c.hits + 65536));
  }

  // Every capacity-dependent buffer with the bytes capacities c need: f(buffer, bytes).
  template <typename F>
  void for_buffers(const Caps& c, F&& f) {
    const size_t nm = geo->nm;
    f(sen_cnt, std::max<size_t>(c.ev * 2 * nm + 1, 1) * sizeof(uint32_t));
    f(sen_off, std::max<size_t>(c.ev * 2 * nm + 1, 1) * sizeof(uint32_t));
    f(hit_tmp, std::max<size_t>(c.hits, 1) * sizeof(uint32_t));
    f(hit_psi, std::max<size_t>(c.hits, 1) * sizeof(float));
    f(hit_ev, std::max<size_t>(c.hits, 1) * sizeof(uint32_t));
    f(hit_idx, std::max<size_t>(c.hits, 1) * sizeof(uint32_t));
    f(hit_sen, std::max<size_t>(c.hits, 1) * sizeof(uint32_t));
    f(hit4, std::max<size_t>(c.hits, 1) * sizeof(float4));
    f(md_hcnt, std::max<size_t>(c.hits, 1) * sizeof(uint32_t));
    f(md_hoff, std::max<size_t>(c.hits + 1, 1) * sizeof(uint32_t));
    f(md_hmask, std::max<size_t>(c.hits, 1) * sizeof(uint32_t));
    f(md_off, std::max<size_t>(c.ev * nm + 1, 1) * sizeof(uint32_t));
    f(md_box, std::max<size_t>(2 * (size_t)c.ev * nm, 1) * sizeof(float4));
    f(md_unit, std::max<size_t>(c.md, 1) * sizeof(uint32_t));
    f(md_lo_idx, std::max<size_t>(c.md, 1) * sizeof(uint32_t));
    f(md_up_idx, std::max<size_t>(c.md, 1) * sizeof(uint32_t));
    f(md_pt, std::max<size_t>(2 * c.md, 1) * sizeof(float4));
    f(md_up4, std::max<size_t>(c.md, 1) * sizeof(float4));
    f(md_dir4, std::max<size_t>(c.md, 1) * sizeof(float4));
    f(md_psi, std::max<size_t>(c.md, 1) * sizeof(float));
    f(ls_cnt, std::max<size_t>(c.md, 1) * sizeof(uint32_t));
    f(ls_off, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(ls_in, std::max<size_t>(c.ls, 1) * sizeof(uint32_t));
    f(ls_out, std::max<size_t>(c.ls, 1) * sizeof(uint32_t));
    f(t3_lcnt, std::max<size_t>(c.ls, 1) * sizeof(uint32_t));
    f(t3_mask, std::max<size_t>(c.ls, 1) * sizeof(uint32_t));
    f(t3_loff, std::max<size_t>(c.ls + 1, 1) * sizeof(uint32_t));
    f(t3_off, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(t3_a, std::max<size_t>(c.t3, 1) * sizeof(uint32_t));
    f(t3_md4, std::max<size_t>(c.t3, 1) * sizeof(uint4));
    f(t3_b, std::max<size_t>(c.t3, 1) * sizeof(uint32_t));
    f(t3_c, std::max<size_t>(c.t3, 1) * sizeof(uint32_t));
    f(t5_tcnt, std::max<size_t>(c.t3, 1) * sizeof(uint32_t));
    f(t5_mask, std::max<size_t>(c.t3, 1) * sizeof(uint32_t));
    f(t5_toff, std::max<size_t>(c.t3 + 1, 1) * sizeof(uint32_t));
    f(t5_off, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    for (auto& b : t5_m) f(b, std::max<size_t>(c.t5, 1) * sizeof(uint32_t));
    f(t5_score, std::max<size_t>(c.t5, 1) * sizeof(float));
    f(t5_md8, std::max<size_t>(2 * (size_t)c.t5, 1) * sizeof(uint4));
    f(t5_kfull, std::max<size_t>(c.t5, 1) * sizeof(float));
    f(pls_ev, std::max<size_t>(c.pls, 1) * sizeof(uint32_t));
    f(pls_ncand, std::max<size_t>(c.pls, 1) * sizeof(uint32_t));
    f(pls_cand, std::max<size_t>((size_t)c.pls * MAX_CAND, 1) * sizeof(uint32_t));
    f(pls_mdpass, std::max<size_t>((size_t)c.pls * PLS_MD_CAP, 1) * sizeof(uint32_t));
    f(pls_nmdpass, std::max<size_t>(c.pls, 1) * sizeof(uint32_t));
    f(pls_h0, std::max<size_t>(c.pls, 1) * sizeof(float4));
    f(pls_h1, std::max<size_t>(c.pls, 1) * sizeof(float4));
    f(pls_pt, std::max<size_t>(c.pls, 1) * sizeof(float));
    f(pt3_icnt, std::max<size_t>(c.pls, 1) * sizeof(uint32_t));
    f(pt3_ioff, std::max<size_t>(c.pls + 1, 1) * sizeof(uint32_t));
    f(pt3_item_p, std::max<size_t>((size_t)c.pls * PLS_ITEMS, 1) * sizeof(uint32_t));
    f(pt3_xcnt, std::max<size_t>((size_t)c.pls * PLS_ITEMS, 1) * sizeof(uint32_t));
    f(pt3_xoff, std::max<size_t>((size_t)c.pls * PLS_ITEMS + 1, 1) * sizeof(uint32_t));
    f(pt3_xmask, std::max<size_t>((size_t)c.pls * PLS_ITEMS, 1) * sizeof(uint32_t));
    f(pt3_off, std::max<size_t>(c.pls + 1, 1) * sizeof(uint32_t));
    f(pt3_pls, std::max<size_t>(c.pt3, 1) * sizeof(uint32_t));
    f(pt3_obj, std::max<size_t>(c.pt3, 1) * sizeof(uint32_t));
    f(pt3_score, std::max<size_t>(c.pt3, 1) * sizeof(float));
    f(pt5_xcnt, std::max<size_t>(c.pt3, 1) * sizeof(uint32_t));
    f(pt5_xoff, std::max<size_t>(c.pt3 + 1, 1) * sizeof(uint32_t));
    f(pt5_xmask, std::max<size_t>(c.pt3, 1) * sizeof(uint32_t));
    f(pt5_off, std::max<size_t>(c.pls + 1, 1) * sizeof(uint32_t));
    f(pt5_pls, std::max<size_t>(c.pt5, 1) * sizeof(uint32_t));
    f(pt5_obj, std::max<size_t>(c.pt5, 1) * sizeof(uint32_t));
    f(pt5_score, std::max<size_t>(c.pt5, 1) * sizeof(float));
    f(c5_cnt, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(c5_off, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(c5_list, std::max<size_t>((size_t)5 * c.pt5, 1) * sizeof(uint32_t));
    f(c3_cnt, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(c3_off, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(c3_list, std::max<size_t>((size_t)3 * c.pt3, 1) * sizeof(uint32_t));
    f(ct_cnt, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(ct_off, std::max<size_t>(c.md + 1, 1) * sizeof(uint32_t));
    f(ct_list, std::max<size_t>((size_t)5 * c.t5, 1) * sizeof(uint32_t));
    f(alive5, std::max<size_t>(c.pt5, 1) * sizeof(uint32_t));
    f(alive3, std::max<size_t>(c.pt3, 1) * sizeof(uint32_t));
    f(alivet, std::max<size_t>(c.t5, 1) * sizeof(uint32_t));
    f(plstc, std::max<size_t>(c.pls, 1) * sizeof(uint32_t));
    f(cross3, std::max<size_t>(c.pt3, 1) * sizeof(uint32_t));
    f(crosst, std::max<size_t>(c.t5, 1) * sizeof(uint32_t));
    f(sa5, std::max<size_t>(c.pt5 + 1, 1) * sizeof(uint32_t));
    f(sa3, std::max<size_t>(c.pt3 + 1, 1) * sizeof(uint32_t));
    f(sat, std::max<size_t>(c.t5 + 1, 1) * sizeof(uint32_t));
    f(sap, std::max<size_t>(c.pls + 1, 1) * sizeof(uint32_t));
    f(tc_ev_off, std::max<size_t>(c.ev + 1, 1) * sizeof(uint32_t));
    f(tc, std::max<size_t>(c.tc, 1) * sizeof(lst_tc));
    f(mask_off, std::max<size_t>(c.md, 1) * sizeof(uint32_t));
    f(mask, (size_t)mask_words(c) * sizeof(uint32_t));
    f(scan_state, (size_t)N_SCAN_SLOTS * scan_chunks_for(c) * sizeof(unsigned long long));
  }

  // Chunks of the largest array a scan of the chain may hold at capacities c (the bound each
  // scan is launched with), hence the chunk states one scan slot needs.
  uint32_t scan_chunks_for(const Caps& c) const {
    const uint64_t b = std::max<uint64_t>(
        {(uint64_t)c.ev * 2 * geo->nm, c.hits, c.md, c.ls, c.t3, c.t5, c.pt3, c.pt5, (uint64_t)c.pls * PLS_ITEMS});
    return (uint32_t)std::max<uint64_t>(1, (b + SCAN_LARGE_CHUNK - 1) / SCAN_LARGE_CHUNK);
  }

  // Clears the chunk states (a new array may hold anything, and after 2^30 - 1 runs the tags
  // repeat), ordered before whatever is launched next on s.
  void clear_scan_state(cudaStream_t s) {
    CK(cudaMemsetAsync(scan_state.p, 0, scan_state.bytes, s));
    CK(cudaStreamSynchronize(s));
  }

  // Grow every buffer to the capacities in c (never shrinks).
  void ensure_caps(const Caps& c_in) {
    const Caps c = merged(c_in);
    const uint32_t words = mask_words(c);
    const void* state_before = scan_state.p;
    for_buffers(c, [&](DevBuf& b, size_t bytes) {
      const size_t before = b.bytes;
      b.ensure(bytes, dev_bytes);
      if (b.bytes != before) graph_valid = false;
    });
    scan_chunks = scan_chunks_for(c);
    if (scan_state.p != state_before) clear_scan_state(stream);
    cap_mask = words;
    cap = c;
  }

  // Device bytes the pipeline would hold after ensure_caps(c) and ensure_inputs(ne, nh, np),
  // without allocating anything (serving admission under a memory budget).
  uint64_t bytes_after(const Caps& c_in, uint32_t ne, uint32_t nh, uint32_t np) {
    uint64_t t = dev_bytes;
    auto add = [&](const DevBuf& b, size_t bytes) {
      if (bytes > b.bytes) t += bytes - b.bytes;
    };
    for_buffers(merged(c_in), add);
    add(in_x, std::max<size_t>(nh, 1) * 4);
    add(in_y, std::max<size_t>(nh, 1) * 4);
    add(in_z, std::max<size_t>(nh, 1) * 4);
    add(in_det, std::max<size_t>(nh, 1) * 4);
    add(in_hoff, (size_t)(ne + 1) * 4);
    add(in_pls, std::max<size_t>(np, 1) * sizeof(PlsIn));
    add(in_poff, (size_t)(ne + 1) * 4);
    return t;
  }

  // Grows the LS partner-list arena to what the last run used (words handed out up to the
  // arena's end plus the exact needs of the lists that found it exhausted), with 25 %
  // headroom; under a byte cap (a serving slot's budget share) it grows only as far as the
  // cap allows -- a smaller arena only means more anchors joined again by the fill pass.
  void learn_mask(const Hdr& h) {
    const uint64_t used = std::min<uint64_t>(h.mask_used[1], cap_mask) + h.mask_used[2];
    if (used <= cap_mask || test_mask_words) return;
    uint64_t want = std::min<uint64_t>(4000000000ull, used * 5 / 4 + 65536);
    if (byte_cap) {
      const uint64_t others = dev_bytes - mask.bytes;
      const uint64_t room = byte_cap > others ? (byte_cap - others) / sizeof(uint32_t) : 0;
      want = std::min(want, room);
    }
    if (want > cap_mask) {
      need<uint32_t>(mask, (size_t)want);
      cap_mask = (uint32_t)want;
    }
  }

  void ensure_inputs(uint32_t ne, uint32_t nh, uint32_t np) {
    need<float>(in_x, nh);
    need<float>(in_y, nh);
    need<float>(in_z, nh);
    need<uint32_t>(in_det, nh);
    need<uint32_t>(in_hoff, ne + 1);
    need<PlsIn>(in_pls, np);
    need<uint32_t>(in_poff, ne + 1);
  }

  Caps estimate(uint32_t ne, uint32_t nh, uint32_t np) const {
    Caps c;
    c.ev = ne;
    c.hits = nh;
    c.pls = np;
    auto f = [](double r, uint32_t n) { return (uint32_t)std::min(4.0e9, r * n * 1.25 + 1024); };
    c.md = f(r_md, nh);
    c.ls = f(r_ls, nh);
    c.t3 = f(r_t3, nh);
    c.t5 = f(r_t5, nh);
    c.pt3 = f(r_pt3, np);
    c.pt5 = f(r_pt5, np);
    c.tc = c.t5 + np + 1024;
    return c;
  }

  // Learn sizes from a finished run so that the next estimate is large enough.
  void learn(const Hdr& h) {
    learn_mask(h);
    // a neighbour list longer than the LS pass's shared-memory list sent its module to the
    // per-MD join: later runs get a list that holds it, up to LS_LIST_MAX (when the cap is
    // the library's choice; a shorter list keeps more blocks resident, so 512 stays the start)
    if (h.ls_maxlen > L.ls_list_cap && auto_list_cap && L.ls_list_cap && L.ls_list_cap < LS_LIST_MAX) {
      L.ls_list_cap = std::min(LS_LIST_MAX, (h.ls_maxlen + 127u) & ~127u);
      graph_valid = false;
    }
    if (h.n_hits) {
      r_md = std::max(r_md, (double)h.tot[T_MD] / h.n_hits);
      r_ls = std::max(r_ls, (double)h.tot[T_LS] / h.n_hits);
      r_t3 = std::max(r_t3, (double)h.tot[T_T3] / h.n_hits);
      r_t5 = std::max(r_t5, (double)h.tot[T_T5] / h.n_hits);
    }
    if (h.n_pls) {
      r_pt3 = std::max(r_pt3, (double)h.tot[T_PT3] / h.n_pls);
      r_pt5 = std::max(r_pt5, (double)h.tot[T_PT5] / h.n_pls);
    }
  }

  BufView view() {
    BufView v;
    v.hdr = (Hdr*)hdr.p;
    v.cap_ev = cap.ev; v.cap_hits = cap.hits; v.cap_md = cap.md; v.cap_ls = cap.ls; v.cap_t3 = cap.t3;
    v.cap_t5 = cap.t5; v.cap_pls = cap.pls; v.cap_pt3 = cap.pt3; v.cap_pt5 = cap.pt5; v.cap_tc = cap.tc;
#define P32(x) (uint32_t*)x.p
    v.sen_cnt = P32(sen_cnt); v.sen_off = P32(sen_off); v.hit_tmp = P32(hit_tmp); v.hit_psi = (float*)hit_psi.p; v.hit_ev = P32(hit_ev);
    v.hit_idx = P32(hit_idx); v.hit4 = (float4*)hit4.p;
    v.md_hcnt = P32(md_hcnt); v.md_hoff = P32(md_hoff); v.md_hmask = P32(md_hmask); v.md_box = (float4*)md_box.p; v.hit_sen = P32(hit_sen); v.md_off = P32(md_off); v.md_unit = P32(md_unit); v.md_lo_idx = P32(md_lo_idx);
    v.md_up_idx = P32(md_up_idx); v.md_pt = (float4*)md_pt.p; v.md_up4 = (float4*)md_up4.p;
    v.md_dir4 = (float4*)md_dir4.p;
    v.md_psi = (float*)md_psi.p;
    v.ls_cnt = P32(ls_cnt); v.ls_off = P32(ls_off); v.ls_in = P32(ls_in); v.ls_out = P32(ls_out);
    v.t3_lcnt = P32(t3_lcnt); v.t3_loff = P32(t3_loff); v.t3_off = P32(t3_off); v.t3_mask = P32(t3_mask);
    v.t3_a = P32(t3_a); v.t3_b = P32(t3_b); v.t3_c = P32(t3_c); v.t3_md4 = (uint4*)t3_md4.p;
    v.t5_tcnt = P32(t5_tcnt); v.t5_toff = P32(t5_toff); v.t5_off = P32(t5_off); v.t5_mask = P32(t5_mask);
    v.t5_m0 = P32(t5_m[0]); v.t5_m1 = P32(t5_m[1]); v.t5_m2 = P32(t5_m[2]); v.t5_m3 = P32(t5_m[3]);
    v.t5_md8 = (uint4*)t5_md8.p;
    v.t5_m4 = P32(t5_m[4]);
    v.t5_score = (float*)t5_score.p; v.t5_kfull = (float*)t5_kfull.p;
    v.pls_ev = P32(pls_ev); v.pls_ncand = P32(pls_ncand); v.pls_cand = P32(pls_cand);
    v.pls_mdpass = P32(pls_mdpass); v.pls_nmdpass = P32(pls_nmdpass);
    v.pls_h0 = (float4*)pls_h0.p; v.pls_h1 = (float4*)pls_h1.p; v.pls_pt = (float*)pls_pt.p;
    v.pt3_icnt = P32(pt3_icnt); v.pt3_ioff = P32(pt3_ioff); v.pt3_item_p = P32(pt3_item_p);
    v.pt3_xcnt = P32(pt3_xcnt); v.pt3_xoff = P32(pt3_xoff); v.pt3_xmask = P32(pt3_xmask); v.pt3_off = P32(pt3_off); v.pt3_pls = P32(pt3_pls); v.pt3_obj = P32(pt3_obj);
    v.pt3_score = (float*)pt3_score.p;
    v.pt5_xcnt = P32(pt5_xcnt); v.pt5_xoff = P32(pt5_xoff); v.pt5_xmask = P32(pt5_xmask); v.pt5_off = P32(pt5_off); v.pt5_pls = P32(pt5_pls); v.pt5_obj = P32(pt5_obj);
    v.pt5_score = (float*)pt5_score.p;
    v.c5_cnt = P32(c5_cnt); v.c5_off = P32(c5_off); v.c5_list = P32(c5_list);
    v.c3_cnt = P32(c3_cnt); v.c3_off = P32(c3_off); v.c3_list = P32(c3_list);
    v.ct_cnt = P32(ct_cnt); v.ct_off = P32(ct_off); v.ct_list = P32(ct_list);
    v.alive5 = P32(alive5); v.alive3 = P32(alive3); v.alivet = P32(alivet); v.plstc = P32(plstc);
    v.cross3 = P32(cross3); v.crosst = P32(crosst);
    v.sa5 = P32(sa5); v.sa3 = P32(sa3); v.sat = P32(sat); v.sap = P32(sap);
    v.tc_ev_off = P32(tc_ev_off); v.tc = tc.p;
    v.mask = P32(mask); v.mask_off = P32(mask_off); v.cap_mask = cap_mask;
    v.scan_state = (unsigned long long*)scan_state.p; v.scan_chunks = scan_chunks;
#undef P32
    return v;
  }

  static void mark_cb(void* arg, int name) {
    Pipeline* P = (Pipeline*)arg;
    const size_t k = P->prof_name.size();
    if (k < P->prof_ev.size()) {
      cudaEventRecord(P->prof_ev[k], P->cur_stream);
      P->prof_name.push_back(name);
    }
  }
  cudaStream_t cur_stream = nullptr;

  // Enqueue header upload, the kernels and the header read-back (eagerly or as one graph)
  // on stream `on` (null: the pipeline's own stream).
  // after (may be null): an event the chain must wait for (another slot's batch) -- the
  // inputs already uploaded on this stream are not held back by it
  void launch(bool use_graph, cudaStream_t on = nullptr, cudaEvent_t after = nullptr) {
    // every kernel writes per-event and per-hit arrays: never launch before ensure_caps sized
    // them for this batch
    if (cap.ev < dev_inputs.n_ev || cap.hits < dev_inputs.n_hits || cap.pls < dev_inputs.n_pls || cap.ev == 0)
      throw StatusError{LST_ERR_INVALID_ARG, "internal: pipeline launched before its buffers were sized"};
    *h_hdr = dev_inputs;
    if (epoch == 0x3FFFFFFFu) {  // the 30-bit run tags would repeat: start again from clear states
      clear_scan_state(on ? on : stream);
      epoch = 0;
    }
    h_hdr->scan_epoch = ++epoch;
    if (stall_scan_runs) {
      stall_scan_runs--;
      for (uint32_t& t : h_hdr->scan_ticket) t = 1;  // no block takes chunk 0
    }
    L.t5_mlp = geo->has_t5_mlp ? &geo->t5_mlp : nullptr;
    if (graph_sel_version != geo->sel_version) {
      graph_valid = false;
      graph_sel_version = geo->sel_version;
    }
    const GeoView G = geo->view();
    const BufView B = view();
    cudaStream_t st = on ? on : stream;
    cur_stream = st;
    if (after) CK(cudaStreamWaitEvent(st, after, 0));
    if (profile) {
      prof_name.clear();
      CK(cudaMemcpyAsync(hdr.p, h_hdr, sizeof(Hdr), cudaMemcpyHostToDevice, st));
      CK(cudaEventRecord(prof_start, st));
      kernels = enqueue_pipeline(C, G, B, L, st, &Pipeline::mark_cb, this);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h_hdr_out, hdr.p, sizeof(Hdr), cudaMemcpyDeviceToHost, st));
      CK(cudaEventRecord(done, st));
      return;
    }
    if (use_graph) {
      if (!graph_valid) {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        cudaMemcpyAsync(hdr.p, h_hdr, sizeof(Hdr), cudaMemcpyHostToDevice, stream);
        kernels = enqueue_pipeline(C, G, B, L, stream, nullptr, nullptr, &side);
        cudaMemcpyAsync(h_hdr_out, hdr.p, sizeof(Hdr), cudaMemcpyDeviceToHost, stream);
        CK(cudaStreamEndCapture(stream, &g));
        cudaError_t e = cudaGraphInstantiate(&graph, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        graph_valid = true;
      }
      CK(cudaGraphLaunch(graph, st));
    } else {
      CK(cudaMemcpyAsync(hdr.p, h_hdr, sizeof(Hdr), cudaMemcpyHostToDevice, st));
      kernels = enqueue_pipeline(C, G, B, L, st, nullptr, nullptr, &side);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h_hdr_out, hdr.p, sizeof(Hdr), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaEventRecord(done, st));
  }

  // Per-kernel times of the last profiled run, summed by kernel name.
  std::vector<lst_profile_entry> profile_entries() {
    std::vector<lst_profile_entry> out;
    if (!profile) return out;
    std::map<int, std::pair<uint32_t, float>> acc;
    cudaEvent_t prev = prof_start;
    for (size_t k = 0; k < prof_name.size(); k++) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, prev, prof_ev[k]));
      auto& a = acc[prof_name[k]];
      a.first += 1;
      a.second += ms;
      prev = prof_ev[k];
    }
    for (auto& kv : acc) {
      lst_profile_entry e{};
      snprintf(e.name, sizeof(e.name), "%s", kKernelNames[kv.first]);
      e.launches = kv.second.first;
      e.ms = kv.second.second;
      out.push_back(e);
    }
    return out;
  }

  // Bounded wait for the launched batch; false on timeout.
  bool wait(uint32_t timeout_ms) {
    if (timeout_ms == 0) {
      CK(cudaEventSynchronize(done));
      return true;
    }
    const double t_end = now_s() + timeout_ms * 1e-3;
    for (;;) {
      const cudaError_t e = cudaEventQuery(done);
      if (e == cudaSuccess) return true;
      if (e != cudaErrorNotReady) throw CudaError{e, "cudaEventQuery"};
      if (now_s() > t_end) return false;
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }

  // Grow whatever overflowed (from the header) and report whether a re-run is needed.
  bool grow_after_overflow(const Hdr& h) {
    const uint32_t bits = h.err >> ERR_OVERFLOW_SHIFT;
    if (!bits) return false;
    Caps c = cap;
    auto g = [](uint32_t need) { return (uint32_t)std::min<uint64_t>(4000000000ull, (uint64_t)need * 5 / 4 + 4096); };
    if (bits & (1u << T_MD)) c.md = g(h.tot[T_MD]);
    if (bits & (1u << T_LS)) c.ls = g(h.tot[T_LS]);
    if (bits & (1u << T_T3)) c.t3 = g(h.tot[T_T3]);
    if (bits & (1u << T_T5)) c.t5 = g(h.tot[T_T5]);
    if (bits & (1u << T_PT3)) c.pt3 = g(h.tot[T_PT3]);
    if (bits & (1u << T_PT5)) c.pt5 = g(h.tot[T_PT5]);
    if (bits & (1u << T_C5)) c.pt5 = g(h.tot[T_C5] / 5 + 1);
    if (bits & (1u << T_C3)) c.pt3 = g(h.tot[T_C3] / 3 + 1);
    if (bits & (1u << T_CT)) c.t5 = g(h.tot[T_CT] / 5 + 1);
    if (bits & (1u << T_TC)) c.tc = g(h.tot[T_TC]);
    ensure_caps(c);
    return true;
  }
};

void pack_host_events(Pipeline& P, const lst_event* evs, uint32_t n) {
  uint64_t nh = 0, np = 0;
  for (uint32_t i = 0; i < n; i++) {
    if ((!evs[i].x || !evs[i].y || !evs[i].z || !evs[i].det) && evs[i].n_hits)
      throw StatusError{LST_ERR_INVALID_ARG, "event with null hit arrays"};
    if (!evs[i].pls && evs[i].n_pls) throw StatusError{LST_ERR_INVALID_ARG, "event with null pLS array"};
    nh += evs[i].n_hits;
    np += evs[i].n_pls;
  }
  if (nh > 0xF0000000ull || np > 0x0F000000ull) throw StatusError{LST_ERR_INVALID_ARG, "batch too large"};
  P.ensure_inputs(n, (uint32_t)nh, (uint32_t)np);
  const size_t bytes = nh * 16 + np * sizeof(PlsIn) + 2 * (n + 1) * 4 + 64;
  if (bytes > P.h_stage_bytes) {
    if (P.h_stage) cudaFreeHost(P.h_stage);
    P.h_stage = nullptr;
    P.h_stage_bytes = 0;
    CK(cudaMallocHost(&P.h_stage, bytes * 3 / 2));
    P.h_stage_bytes = bytes * 3 / 2;
  }
  char* s = (char*)P.h_stage;
  float* hx = (float*)s;
  float* hy = hx + nh;
  float* hz = hy + nh;
  uint32_t* hd = (uint32_t*)(hz + nh);
  uint32_t* hoff = hd + nh;
  uint32_t* poff = hoff + (n + 1);
  PlsIn* hp = (PlsIn*)(((uintptr_t)(poff + n + 1) + 15) & ~(uintptr_t)15);
  uint64_t oh = 0, op = 0;
  for (uint32_t i = 0; i < n; i++) {
    hoff[i] = (uint32_t)oh;
    poff[i] = (uint32_t)op;
    oh += evs[i].n_hits;
    op += evs[i].n_pls;
  }
  hoff[n] = (uint32_t)oh;
  poff[n] = (uint32_t)op;
  // copy the events into the pinned staging area, on several host threads for big batches
  auto copy_range = [&](uint32_t e0, uint32_t e1) {
    for (uint32_t i = e0; i < e1; i++) {
      const lst_event& e = evs[i];
      if (e.n_hits) {
        memcpy(hx + hoff[i], e.x, e.n_hits * 4);
        memcpy(hy + hoff[i], e.y, e.n_hits * 4);
        memcpy(hz + hoff[i], e.z, e.n_hits * 4);
        memcpy(hd + hoff[i], e.det, e.n_hits * 4);
      }
      if (e.n_pls) memcpy(hp + poff[i], e.pls, e.n_pls * sizeof(PlsIn));
    }
  };
  const uint64_t total_bytes = nh * 16 + np * sizeof(PlsIn);
  const uint32_t nt = (uint32_t)std::min<uint64_t>({(uint64_t)n, 16u, total_bytes / (1u << 20) + 1});
  if (nt <= 1) {
    copy_range(0, n);
  } else {
    // split events into nt ranges of about equal bytes, copied by the pipeline's helpers
    std::vector<uint32_t> cut(nt + 1, n);
    cut[0] = 0;
    uint64_t acc = 0;
    uint32_t k = 1;
    for (uint32_t i = 0; i < n && k < nt; i++) {
      acc += (uint64_t)evs[i].n_hits * 16 + (uint64_t)evs[i].n_pls * sizeof(PlsIn);
      if (acc * nt >= total_bytes * k) cut[k++] = i + 1;
    }
    P.copiers().run(nt, [&](uint32_t t) { copy_range(cut[t], cut[t + 1]); });
  }
  cudaStream_t st = P.stream;
  if (nh) {
    CK(cudaMemcpyAsync(P.in_x.p, hx, nh * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P.in_y.p, hy, nh * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P.in_z.p, hz, nh * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P.in_det.p, hd, nh * 4, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(P.in_hoff.p, hoff, (n + 1) * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(P.in_poff.p, poff, (n + 1) * 4, cudaMemcpyHostToDevice, st));
  if (np) CK(cudaMemcpyAsync(P.in_pls.p, hp, np * sizeof(PlsIn), cudaMemcpyHostToDevice, st));
  Hdr h{};
  h.x = (const float*)P.in_x.p;
  h.y = (const float*)P.in_y.p;
  h.z = (const float*)P.in_z.p;
  h.det = (const uint32_t*)P.in_det.p;
  h.hit_off = (const uint32_t*)P.in_hoff.p;
  h.pls = (const PlsIn*)P.in_pls.p;
  h.pls_off = (const uint32_t*)P.in_poff.p;
  h.n_ev = n;
  h.n_hits = (uint32_t)nh;
  h.n_pls = (uint32_t)np;
  P.dev_inputs = h;
  P.n_ev = n;
  P.n_hits = (uint32_t)nh;
  P.n_pls = (uint32_t)np;
}

}  // namespace

// ------------------------------------------------------------------ context
struct lst_ctx {
  std::mutex mu;  // results, statistics and the error text (the serving workers share them)
  lst_config cfg{};
  int device = 0;
  int n_sm = 0;
  Geometry geo;
  Pipeline main;
  std::map<lst_result_id, Result> results;
  lst_result_id next_id = 1;
  std::string err;
  lst_stats stats{};
  uint32_t reruns = 0;
  std::unique_ptr<Workers> getters;  // copies for lst_get_candidates_batch (used under mu only)
  // lst_submit_batch / lst_collect_batch: two slots, each with its own pipeline
  struct AsyncSlot {
    std::unique_ptr<Pipeline> P;
    uint64_t ticket = 0;  // 0: free
    uint32_t n_ev = 0;
  };
  AsyncSlot slots[2];
  uint64_t next_ticket = 1;
  // last lst_serve_replay: batches launched, largest batch, peak device bytes
  uint32_t served_batches = 0, served_max_batch = 0;
  uint64_t served_peak_bytes = 0;
};

namespace {

lst_status fail(lst_ctx* c, lst_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

template <typename F>
lst_status guarded(lst_ctx* c, F&& f) {
  try {
    if (c) cudaSetDevice(c->device);
    return f();
  } catch (const CudaError& e) {
    return fail(c, LST_ERR_CUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
  } catch (const StatusError& e) {
    return fail(c, e.s, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(c, LST_ERR_OOM, "host allocation failed");
  }
}

// Copy the per-event results of a finished batch to the host.
void collect(lst_ctx* c, Pipeline& P, lst_result_id* outs, uint32_t* n_tc_per_event) {
  const Hdr& h = *P.h_hdr_out;
  const uint32_t ne = P.n_ev;
  std::vector<uint32_t> evoff(ne + 1);
  CK(cudaMemcpyAsync(evoff.data(), P.tc_ev_off.p, (ne + 1) * 4, cudaMemcpyDeviceToHost, P.stream));
  // candidates: device -> pinned landing area (fast), then copied by the helpers into one
  // buffer shared by the batch's results
  const size_t n_tc = outs ? h.tot[T_TC] : 0;
  if (n_tc > P.h_tc_cap) {
    if (P.h_tc) cudaFreeHost(P.h_tc);
    P.h_tc = nullptr;
    P.h_tc_cap = 0;
    CK(cudaMallocHost((void**)&P.h_tc, n_tc * 3 / 2 * sizeof(lst_tc)));
    P.h_tc_cap = n_tc * 3 / 2;
  }
  if (n_tc) CK(cudaMemcpyAsync(P.h_tc, P.tc.p, n_tc * sizeof(lst_tc), cudaMemcpyDeviceToHost, P.stream));
  const bool keep = c->cfg.keep_objects != 0 && outs;
  std::vector<uint32_t> md_off, md_unit, md_lo, md_up, ls_in, ls_out, t3a, t3b, t3c, t5m[5], t3_off, t5_off, pt3p,
      pt3o, pt5p, pt5o, a5, a3, at, ptc, pncand, pcand, pt3_off, pt5_off, poff;
  std::vector<float> t5s, t5k, pt3s, pt5s;
  auto get = [&](auto& v, DevBuf& b, size_t n) {
    v.resize(n);
    if (n) CK(cudaMemcpyAsync(v.data(), b.p, n * sizeof(v[0]), cudaMemcpyDeviceToHost, P.stream));
  };
  if (keep) {
    const size_t nm = c->geo.nm;
    get(md_off, P.md_off, ne * nm + 1);
    get(md_unit, P.md_unit, h.tot[T_MD]);
    get(md_lo, P.md_lo_idx, h.tot[T_MD]);
    get(md_up, P.md_up_idx, h.tot[T_MD]);
    get(ls_in, P.ls_in, h.tot[T_LS]);
    get(ls_out, P.ls_out, h.tot[T_LS]);
    get(t3a, P.t3_a, h.tot[T_T3]);
    get(t3b, P.t3_b, h.tot[T_T3]);
    get(t3c, P.t3_c, h.tot[T_T3]);
    for (int k = 0; k < 5; k++) get(t5m[k], P.t5_m[k], h.tot[T_T5]);
    get(t5s, P.t5_score, h.tot[T_T5]);
    get(t5k, P.t5_kfull, h.tot[T_T5]);
    get(t3_off, P.t3_off, h.tot[T_MD] + 1);
    get(t5_off, P.t5_off, h.tot[T_MD] + 1);
    get(pt3p, P.pt3_pls, h.tot[T_PT3]);
    get(pt3o, P.pt3_obj, h.tot[T_PT3]);
    get(pt3s, P.pt3_score, h.tot[T_PT3]);
    get(pt5p, P.pt5_pls, h.tot[T_PT5]);
    get(pt5o, P.pt5_obj, h.tot[T_PT5]);
    get(pt5s, P.pt5_score, h.tot[T_PT5]);
    get(a5, P.alive5, h.tot[T_PT5]);
    get(a3, P.alive3, h.tot[T_PT3]);
    get(at, P.alivet, h.tot[T_T5]);
    get(ptc, P.plstc, P.n_pls);
    get(pncand, P.pls_ncand, P.n_pls);
    get(pcand, P.pls_cand, (size_t)P.n_pls * MAX_CAND);
    get(pt3_off, P.pt3_off, P.n_pls + 1);
    get(pt5_off, P.pt5_off, P.n_pls + 1);
    get(poff, P.in_poff, ne + 1);
  }
  CK(cudaStreamSynchronize(P.stream));
  std::shared_ptr<lst_tc[]> tcs_ptr(new lst_tc[n_tc ? n_tc : 1]);
  if (n_tc) {
    const uint32_t parts = (uint32_t)std::min<size_t>(16, n_tc / 4096 + 1);
    const size_t per = (n_tc + parts - 1) / parts;
    P.copiers().run(parts, [&](uint32_t t) {
      const size_t b = t * per, e = std::min(n_tc, b + per);
      if (b < e) memcpy(tcs_ptr.get() + b, P.h_tc + b, (e - b) * sizeof(lst_tc));
    });
  }
  const uint32_t nm = c->geo.nm;
  for (uint32_t e = 0; e < ne; e++) {
    if (n_tc_per_event) n_tc_per_event[e] = evoff[e + 1] - evoff[e];
    if (!outs) continue;
    Result r;
    r.tc_buf = tcs_ptr;
    r.tc_off = evoff[e];
    r.tc_n = evoff[e + 1] - evoff[e];
    if (keep) {
      r.has_objects = true;
      const uint32_t mb = md_off[(size_t)e * nm], me = md_off[(size_t)(e + 1) * nm];
      for (uint32_t i = mb; i < me; i++) r.md.push_back({md_unit[i] - e * nm, md_lo[i], md_up[i]});
      // LS of this event: those whose inner MD is in [mb, me)
      for (size_t i = 0; i < ls_in.size(); i++)
        if (ls_in[i] >= mb && ls_in[i] < me) r.ls.push_back({{ls_in[i] - mb, ls_out[i] - mb}});
      const uint32_t tb = t3_off[mb], te = t3_off[me];
      for (uint32_t i = tb; i < te; i++) r.t3.push_back({{t3a[i] - mb, t3b[i] - mb, t3c[i] - mb}});
      const uint32_t fb = t5_off[mb], fe = t5_off[me];
      for (uint32_t i = fb; i < fe; i++)
        r.t5.push_back({{t5m[0][i] - mb, t5m[1][i] - mb, t5m[2][i] - mb, t5m[3][i] - mb, t5m[4][i] - mb},
                        t5s[i], t5k[i], at[i]});
      const uint32_t pb = poff[e], pe = poff[e + 1];
      for (uint32_t i = pt3_off[pb]; i < pt3_off[pe]; i++) r.pt3.push_back({pt3p[i] - pb, pt3o[i] - tb, pt3s[i], a3[i]});
      for (uint32_t i = pt5_off[pb]; i < pt5_off[pe]; i++) r.pt5.push_back({pt5p[i] - pb, pt5o[i] - fb, pt5s[i], a5[i]});
      for (uint32_t p = pb; p < pe; p++) {
        lst_pls_rec pr{};
        pr.n_cand = pncand[p];
        for (uint32_t k = 0; k < pr.n_cand && k < MAX_CAND; k++) pr.cand[k] = pcand[(size_t)p * MAX_CAND + k];
        pr.is_tc = ptc[p];
        r.pls.push_back(pr);
      }
    }
    std::lock_guard<std::mutex> lk(c->mu);
    const lst_result_id id = c->next_id++;
    c->results.emplace(id, std::move(r));
    outs[e] = id;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  c->stats.n_events = ne;
  c->stats.n_hits = h.n_hits;
  c->stats.n_pls = h.n_pls;
  c->stats.n_md = h.tot[T_MD];
  c->stats.n_ls = h.tot[T_LS];
  c->stats.n_t3 = h.tot[T_T3];
  c->stats.n_t5 = h.tot[T_T5];
  c->stats.n_pt3 = h.tot[T_PT3];
  c->stats.n_pt5 = h.tot[T_PT5];
  c->stats.n_tc = h.tot[T_TC];
  c->stats.ls_candidates = h.ls_cand;
  c->stats.kernels = (uint32_t)P.kernels;
  c->stats.device_bytes = P.dev_bytes + c->geo.dev_bytes;
}

// Runs the already-packed batch of P to completion: launch, bounded wait, re-run with
// larger buffers while a list overflows.
lst_status run_packed(lst_ctx* c, Pipeline& P, bool use_graph, uint32_t timeout_ms) {
  for (int attempt = 0; attempt < 12; attempt++) {
    P.launch(use_graph);
    if (!P.wait(timeout_ms)) return fail(c, LST_ERR_TIMEOUT, "device did not finish within the time limit");
    const Hdr& h = *P.h_hdr_out;
    if (h.err & ERR_BAD_INPUT)
      return fail(c, LST_ERR_BAD_INPUT, "bad input: module id out of range, non-finite value or invalid pLS");
    if (h.err & ERR_WAIT) return fail(c, LST_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (!P.grow_after_overflow(h)) {
      P.learn(h);
      return LST_OK;
    }
    c->reruns++;
    c->stats.reruns++;
  }
  return fail(c, LST_ERR_OOM, "object lists kept outgrowing their storage");
}

lst_status run_host_batch(lst_ctx* c, const lst_event* evs, uint32_t n, lst_result_id* outs, bool use_graph) {
  if (!c->geo.have_map) return fail(c, LST_ERR_NO_MAP, "lst_build_connection_map has not run");
  Pipeline& P = c->main;
  pack_host_events(P, evs, n);
  P.ensure_caps(P.estimate(n, P.n_hits, P.n_pls));
  const lst_status s = run_packed(c, P, use_graph, 0);
  if (s != LST_OK) return s;
  collect(c, P, outs, nullptr);
  return LST_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* lst_status_string(lst_status s) {
  switch (s) {
    case LST_OK: return "ok";
    case LST_ERR_INVALID_ARG: return "invalid argument";
    case LST_ERR_BAD_INPUT: return "bad input";
    case LST_ERR_NO_MAP: return "connection map not built";
    case LST_ERR_OOM: return "out of memory";
    case LST_ERR_BUDGET: return "memory budget exceeded";
    case LST_ERR_CUDA: return "CUDA error";
    case LST_ERR_TIMEOUT: return "timeout";
    case LST_ERR_BUFFER_TOO_SMALL: return "buffer too small";
    case LST_ERR_NOT_FOUND: return "result not found";
    default: return "unknown status";
  }
}

lst_status lst_load_geometry(const lst_module_desc* mods, uint32_t n_mods, const lst_config* cfg, lst_ctx** out_ctx) {
  if (!mods || n_mods == 0 || !out_ctx) return LST_ERR_INVALID_ARG;
  *out_ctx = nullptr;
  lst_ctx* c = nullptr;
  try {
    c = new lst_ctx();
  } catch (...) {
    return LST_ERR_OOM;
  }
  if (cfg) c->cfg = *cfg;
  c->device = c->cfg.device;
  if ((c->cfg.block_size && (c->cfg.block_size < 64 || c->cfg.block_size > 512 || c->cfg.block_size % 32)) ||
      c->cfg.blocks_per_sm > 32) {
    delete c;
    return LST_ERR_INVALID_ARG;
  }
  const lst_status s = guarded(c, [&]() -> lst_status {
    CK(cudaSetDevice(c->device));
    CK(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device));
    c->geo.load(mods, n_mods);
    c->geo.upload_tables();
    c->main.init(&c->geo, c->cfg, c->n_sm);
    if (const char* v = std::getenv("LST_TEST_STALL_SCAN")) c->main.stall_scan_runs = (uint32_t)std::atoi(v);
    if (const char* v = std::getenv("LST_TEST_MASK_WORDS")) c->main.test_mask_words = (uint32_t)std::atoi(v);
    // test hook: the scans' run tags start at this value (the next run takes it + 1), here
    // and in the allocation-free entry point on this device
    if (const char* v = std::getenv("LST_TEST_SCAN_EPOCH")) {
      const uint32_t e = (uint32_t)std::strtoul(v, nullptr, 0) & 0x3FFFFFFFu;
      c->main.epoch = e;
      static_scan_epoch_set(c->device, e);
    }
    // the allocation-free entry point's array and kernels, loaded now so that its calls allocate nothing
    CK(static_scratch_prepare(c->device));
    return LST_OK;
  });
  if (s != LST_OK) {
    delete c;
    return s;
  }
  *out_ctx = c;
  return LST_OK;
}

lst_status lst_build_connection_map(lst_ctx* c) {
  if (!c) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    c->geo.build_map();
    c->geo.upload_map();
    c->main.graph_valid = false;
    return LST_OK;
  });
}

lst_status lst_run_event(lst_ctx* c, const lst_event* ev, lst_result_id* out) {
  if (!c || !ev || !out) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() { return run_host_batch(c, ev, 1, out, c->cfg.use_graph != 2); });
}

lst_status lst_run_batch(lst_ctx* c, const lst_event* evs, uint32_t n, lst_result_id* outs) {
  if (!c || !evs || !outs || n == 0) return LST_ERR_INVALID_ARG;
  const bool g = c->cfg.use_graph != 2;
  return guarded(c, [&]() { return run_host_batch(c, evs, n, outs, g); });
}

lst_status lst_run_batch_device(lst_ctx* c, const lst_batch_dev* b, void* stream) {
  if (!c || !b || b->n_events == 0 || !b->hit_off || !b->pls_off) return LST_ERR_INVALID_ARG;
  if (b->n_hits && (!b->x || !b->y || !b->z || !b->det)) return LST_ERR_INVALID_ARG;
  if (b->n_pls && !b->pls) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    if (!c->geo.have_map) return fail(c, LST_ERR_NO_MAP, "lst_build_connection_map has not run");
    Pipeline& P = c->main;
    if (P.pending) return fail(c, LST_ERR_INVALID_ARG, "a batch is still in flight (call lst_batch_finish)");
    Hdr h{};
    h.x = b->x; h.y = b->y; h.z = b->z; h.det = b->det; h.hit_off = b->hit_off;
    h.pls = (const PlsIn*)b->pls; h.pls_off = b->pls_off;
    h.n_ev = b->n_events; h.n_hits = b->n_hits; h.n_pls = b->n_pls;
    P.dev_inputs = h;
    P.n_ev = b->n_events;
    P.n_hits = b->n_hits;
    P.n_pls = b->n_pls;
    P.ensure_caps(P.estimate(P.n_ev, P.n_hits, P.n_pls));
    P.launch(c->cfg.use_graph != 2, (cudaStream_t)stream);
    P.pending = true;
    return LST_OK;
  });
}

lst_status lst_batch_finish(lst_ctx* c, uint32_t timeout_ms, uint32_t* n_tc_per_event, lst_result_id* outs) {
  if (!c) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    Pipeline& P = c->main;
    if (!P.pending) return fail(c, LST_ERR_INVALID_ARG, "no batch in flight");
    // on a timeout the batch stays in flight: a later call can wait for it again
    if (!P.wait(timeout_ms)) return fail(c, LST_ERR_TIMEOUT, "device did not finish within the time limit");
    P.pending = false;
    const Hdr& h = *P.h_hdr_out;
    if (h.err & ERR_BAD_INPUT)
      return fail(c, LST_ERR_BAD_INPUT, "bad input: module id out of range, non-finite value or invalid pLS");
    if (h.err & ERR_WAIT) return fail(c, LST_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (P.grow_after_overflow(h)) {
      c->reruns++;
      c->stats.reruns++;
      const lst_status s = run_packed(c, P, c->cfg.use_graph != 2, timeout_ms);
      if (s != LST_OK) return s;
    } else {
      P.learn(h);
    }
    if (n_tc_per_event || outs) collect(c, P, outs, n_tc_per_event);
    return LST_OK;
  });
}

lst_status lst_submit_batch(lst_ctx* c, const lst_event* evs, uint32_t n, uint64_t* ticket) {
  if (!c || !evs || !ticket || n == 0) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    if (!c->geo.have_map) return fail(c, LST_ERR_NO_MAP, "lst_build_connection_map has not run");
    int k = -1;
    for (int i = 0; i < 2 && k < 0; i++)
      if (c->slots[i].ticket == 0) k = i;
    if (k < 0) return fail(c, LST_ERR_INVALID_ARG, "both batch slots are in flight (collect one first)");
    lst_ctx::AsyncSlot& S = c->slots[k];
    lst_ctx::AsyncSlot& other = c->slots[1 - k];
    if (!S.P) {
      S.P.reset(new Pipeline());
      S.P->init(&c->geo, c->cfg, c->n_sm);
    }
    Pipeline& P = *S.P;
    pack_host_events(P, evs, n);  // inputs uploaded on P's stream now
    P.ensure_caps(P.estimate(n, P.n_hits, P.n_pls));
    // the device runs one batch at a time (a batch's working set fills most of the L2):
    // this chain starts when the other slot's finishes
    P.launch(c->cfg.use_graph != 2, nullptr, other.ticket ? other.P->done : nullptr);
    P.pending = true;
    S.ticket = c->next_ticket++;
    S.n_ev = n;
    *ticket = S.ticket;
    return LST_OK;
  });
}

lst_status lst_collect_batch(lst_ctx* c, uint64_t ticket, uint32_t timeout_ms, uint32_t* n_tc_per_event,
                             lst_result_id* outs) {
  if (!c || ticket == 0) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    lst_ctx::AsyncSlot* S = nullptr;
    for (auto& s : c->slots)
      if (s.ticket == ticket) S = &s;
    if (!S) return fail(c, LST_ERR_NOT_FOUND, "unknown or already collected batch ticket");
    Pipeline& P = *S->P;
    // on a timeout the batch stays in flight: a later call can wait for it again
    if (!P.wait(timeout_ms)) return fail(c, LST_ERR_TIMEOUT, "device did not finish within the time limit");
    P.pending = false;
    S->ticket = 0;
    const Hdr& h = *P.h_hdr_out;
    if (h.err & ERR_BAD_INPUT)
      return fail(c, LST_ERR_BAD_INPUT, "bad input: module id out of range, non-finite value or invalid pLS");
    if (h.err & ERR_WAIT) return fail(c, LST_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (P.grow_after_overflow(h)) {
      c->reruns++;
      c->stats.reruns++;
      const lst_status s = run_packed(c, P, c->cfg.use_graph != 2, timeout_ms);
      if (s != LST_OK) return s;
    } else {
      P.learn(h);
    }
    if (n_tc_per_event || outs) collect(c, P, outs, n_tc_per_event);
    return LST_OK;
  });
}

lst_status lst_get_candidates(lst_ctx* c, lst_result_id id, lst_tc* buf, uint32_t cap, uint32_t* n_out) {
  if (!c || !n_out) return LST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->results.find(id);
  if (it == c->results.end()) return fail(c, LST_ERR_NOT_FOUND, "unknown result id");
  const Result& r = it->second;
  *n_out = (uint32_t)r.tc_n;
  if (!buf) return LST_OK;
  if (cap < r.tc_n) return fail(c, LST_ERR_BUFFER_TOO_SMALL, "candidate buffer too small");
  if (r.tc_n) memcpy(buf, r.tc_buf.get() + r.tc_off, r.tc_n * sizeof(lst_tc));
  return LST_OK;
}

// The pLS track candidates (seeds no surviving pT3 or pT5 uses) of a result, as seeds.
lst_status lst_get_seeds(lst_ctx* c, lst_result_id id, int32_t mode, lst_seed* buf, uint32_t cap, uint32_t* n_out) {
  if (!c || !n_out) return LST_ERR_INVALID_ARG;
  if (mode != LST_SEEDS_QUADS && mode != LST_SEEDS_QUADS_TRIPLETS) return fail(c, LST_ERR_INVALID_ARG, "unknown seed mode");
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->results.find(id);
  if (it == c->results.end()) return fail(c, LST_ERR_NOT_FOUND, "unknown result id");
  const Result& r = it->second;
  const lst_tc* tc = r.tc_buf.get() + r.tc_off;
  uint32_t n = 0;
  for (size_t i = 0; i < r.tc_n; i++) {
    if (tc[i].type != LST_TC_PLS || (mode == LST_SEEDS_QUADS && tc[i].n_pix != 4)) continue;
    if (buf) {
      if (n >= cap) return fail(c, LST_ERR_BUFFER_TOO_SMALL, "seed buffer too small");
      buf[n].pls = tc[i].pls;
      buf[n].n_pix = tc[i].n_pix;
      for (int k = 0; k < 4; k++) buf[n].pix[k] = tc[i].pix[k];
    }
    n++;
  }
  *n_out = n;
  return LST_OK;
}

lst_status lst_get_candidates_batch(lst_ctx* c, const lst_result_id* ids, uint32_t n, lst_tc* buf, uint64_t cap,
                                    uint32_t* counts, uint64_t* n_total) {
  if (!c || !n_total || (n && (!ids || !counts))) return LST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  std::vector<const Result*> rs(n);
  uint64_t total = 0;
  for (uint32_t i = 0; i < n; i++) {
    auto it = c->results.find(ids[i]);
    if (it == c->results.end()) return fail(c, LST_ERR_NOT_FOUND, "unknown result id");
    rs[i] = &it->second;
    counts[i] = (uint32_t)rs[i]->tc_n;
    total += rs[i]->tc_n;
  }
  *n_total = total;
  if (!buf) return LST_OK;
  if (cap < total) return fail(c, LST_ERR_BUFFER_TOO_SMALL, "candidate buffer too small");
  std::vector<uint64_t> at(n + 1, 0);
  for (uint32_t i = 0; i < n; i++) at[i + 1] = at[i] + rs[i]->tc_n;
  auto copy = [&](uint32_t i) {
    if (rs[i]->tc_n) memcpy(buf + at[i], rs[i]->tc_buf.get() + rs[i]->tc_off, rs[i]->tc_n * sizeof(lst_tc));
  };
  if (total * sizeof(lst_tc) < (1u << 20) || n < 2) {
    for (uint32_t i = 0; i < n; i++) copy(i);
  } else {  // large: one result per task on the context's helper threads
    if (!c->getters) {
      const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
      c->getters.reset(new Workers(std::min(hw, 16u) - 1));
    }
    c->getters->run(n, copy);
  }
  return LST_OK;
}

lst_status lst_get_objects(lst_ctx* c, lst_result_id id, int32_t kind, void* buf, uint32_t cap, uint32_t* n_out) {
  if (!c || !n_out) return LST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->results.find(id);
  if (it == c->results.end()) return fail(c, LST_ERR_NOT_FOUND, "unknown result id");
  const Result& r = it->second;
  if (!r.has_objects) return fail(c, LST_ERR_INVALID_ARG, "objects were not kept (keep_objects = 0)");
  const void* src = nullptr;
  size_t n = 0, sz = 0;
  switch (kind) {
    case LST_OBJ_MD: src = r.md.data(); n = r.md.size(); sz = sizeof(lst_md_rec); break;
    case LST_OBJ_LS: src = r.ls.data(); n = r.ls.size(); sz = sizeof(lst_ls_rec); break;
    case LST_OBJ_T3: src = r.t3.data(); n = r.t3.size(); sz = sizeof(lst_t3_rec); break;
    case LST_OBJ_T5: src = r.t5.data(); n = r.t5.size(); sz = sizeof(lst_t5_rec); break;
    case LST_OBJ_PT3: src = r.pt3.data(); n = r.pt3.size(); sz = sizeof(lst_px_rec); break;
    case LST_OBJ_PT5: src = r.pt5.data(); n = r.pt5.size(); sz = sizeof(lst_px_rec); break;
    case LST_OBJ_PLS: src = r.pls.data(); n = r.pls.size(); sz = sizeof(lst_pls_rec); break;
    default: return fail(c, LST_ERR_INVALID_ARG, "unknown object kind");
  }
  *n_out = (uint32_t)n;
  if (!buf) return LST_OK;
  if (cap < n) return fail(c, LST_ERR_BUFFER_TOO_SMALL, "object buffer too small");
  if (n) memcpy(buf, src, n * sz);
  return LST_OK;
}

lst_status lst_release_result(lst_ctx* c, lst_result_id id) {
  if (!c) return LST_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->mu);
  if (!c->results.erase(id)) return fail(c, LST_ERR_NOT_FOUND, "unknown result id");
  return LST_OK;
}

void lst_destroy(lst_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  delete c;
}

const char* lst_last_error(lst_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

lst_status lst_set_tuning(lst_ctx* c, const lst_config* cfg) {
  if (!c || !cfg) return LST_ERR_INVALID_ARG;
  const uint32_t bs = cfg->block_size;
  if (bs && (bs < 64 || bs > 512 || bs % 32)) return fail(c, LST_ERR_INVALID_ARG, "block_size must be 64..512, a multiple of 32");
  if (cfg->blocks_per_sm > 32) return fail(c, LST_ERR_INVALID_ARG, "blocks_per_sm must be at most 32");
  return guarded(c, [&]() -> lst_status {
    if (c->main.pending) return fail(c, LST_ERR_INVALID_ARG, "a batch is still in flight");
    c->cfg.block_size = cfg->block_size;
    c->cfg.blocks_per_sm = cfg->blocks_per_sm;
    c->cfg.ls_list_cap = cfg->ls_list_cap;
    c->main.set_tuning(c->cfg, c->n_sm);
    return LST_OK;
  });
}

static_assert(LST_T5_MLP_PARAMS == T5_NPARAM && LST_T5_MLP_INPUTS == T5_NF && LST_T5_MLP_HIDDEN == T5_NH,
              "lst.h and the device network disagree");

lst_status lst_set_t5_selection(lst_ctx* c, const float* weights, uint32_t n) {
  if (!c) return LST_ERR_INVALID_ARG;
  if (weights && n != (uint32_t)T5_NPARAM)
    return fail(c, LST_ERR_INVALID_ARG, "the T5 network takes " + std::to_string(T5_NPARAM) + " weights");
  if (weights)
    for (uint32_t i = 0; i < n; i++)
      if (!std::isfinite(weights[i])) return fail(c, LST_ERR_INVALID_ARG, "T5 network weight " + std::to_string(i) + " is not finite");
  if (c->main.pending || c->slots[0].ticket || c->slots[1].ticket)
    return fail(c, LST_ERR_INVALID_ARG, "a batch is still in flight");
  c->geo.has_t5_mlp = weights != nullptr;
  if (weights) memcpy(c->geo.t5_mlp.w, weights, sizeof(c->geo.t5_mlp.w));
  c->geo.sel_version++;
  return LST_OK;
}

lst_status lst_get_profile(lst_ctx* c, lst_profile_entry* buf, uint32_t cap, uint32_t* n_out) {
  if (!c || !n_out) return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    const std::vector<lst_profile_entry> v = c->main.profile_entries();
    *n_out = (uint32_t)v.size();
    if (!buf) return LST_OK;
    if (cap < v.size()) return fail(c, LST_ERR_BUFFER_TOO_SMALL, "profile buffer too small");
    if (!v.empty()) memcpy(buf, v.data(), v.size() * sizeof(lst_profile_entry));
    return LST_OK;
  });
}

lst_status lst_get_stats(lst_ctx* c, lst_stats* out) {
  if (!c || !out) return LST_ERR_INVALID_ARG;
  *out = c->stats;
  out->reruns = c->reruns;
  out->device_bytes = c->main.dev_bytes + c->geo.dev_bytes;
  out->served_batches = c->served_batches;
  out->served_max_batch = c->served_max_batch;
  out->served_peak_bytes = c->served_peak_bytes;
  out->map_edges = c->geo.conn.size();
  return LST_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ serving
namespace {

struct Slot {
  std::unique_ptr<Pipeline> P;
  std::vector<uint32_t> events;  // indices of the events in flight
  bool busy = false;
};

}  // namespace

extern "C" lst_status lst_serve_replay(lst_ctx* c, const lst_serve_config* cfg, const lst_event* evs,
                                       const double* arrival_s, uint32_t n, double* latency_s, uint32_t* n_tc,
                                       lst_result_id* outs, double* wall_s) {
  if (!c || !cfg || !evs || !arrival_s || n == 0 || !latency_s || cfg->n_slots == 0 || cfg->max_batch == 0)
    return LST_ERR_INVALID_ARG;
  return guarded(c, [&]() -> lst_status {
    if (!c->geo.have_map) return fail(c, LST_ERR_NO_MAP, "lst_build_connection_map has not run");
    std::vector<Slot> slots(cfg->n_slots);
    for (auto& s : slots) {
      s.P.reset(new Pipeline());
      s.P->init(&c->geo, c->cfg, c->n_sm);
      // start from what the main pipeline has learned about object sizes
      s.P->r_md = c->main.r_md; s.P->r_ls = c->main.r_ls; s.P->r_t3 = c->main.r_t3; s.P->r_t5 = c->main.r_t5;
      s.P->r_pt3 = c->main.r_pt3; s.P->r_pt5 = c->main.r_pt5;
    }
    // Memory budget: the context's own buffers stay, the rest is split evenly over the
    // slots; a slot admits events only while its buffers for the batch fit its share.
    const uint64_t budget = cfg->memory_budget;
    const uint64_t base = c->geo.dev_bytes + c->main.dev_bytes;
    if (budget && budget <= base) return fail(c, LST_ERR_BUDGET, "the memory budget is below the context's resident buffers");
    const uint64_t slot_share = budget ? (budget - base) / slots.size() : ~0ull;
    std::atomic<uint32_t> n_batches{0}, max_taken{0};
    std::atomic<uint64_t> peak{0};
    auto fits = [&](Pipeline& P, uint32_t ne, uint64_t nh, uint64_t np) {
      if (!budget) return true;
      if (nh > 0xF0000000ull || np > 0x0F000000ull) return false;
      return P.bytes_after(P.estimate(ne, (uint32_t)nh, (uint32_t)np), ne, (uint32_t)nh, (uint32_t)np) <= slot_share;
    };
    // Before the clock starts: size every slot for the largest batch of typical events (from
    // the first events of the stream) that fits its share, up to max_batch, and capture its graph.
    {
      const uint32_t m = std::min<uint32_t>(n, 64);
      uint64_t sh = 0, sp = 0;
      for (uint32_t i = 0; i < m; i++) {
        sh += evs[i].n_hits;
        sp += evs[i].n_pls;
      }
      auto hits_for = [&](uint32_t b) { return std::min<uint64_t>(0xF0000000ull, sh * 3 / 2 * b / m + 1); };
      auto pls_for = [&](uint32_t b) { return std::min<uint64_t>(0x0F000000ull, sp * 3 / 2 * b / m + 1); };
      uint32_t b = cfg->max_batch;
      while (b > 0 && !fits(*slots[0].P, b, hits_for(b), pls_for(b))) b = b > 8 ? b * 3 / 4 : b - 1;
      for (size_t k = 0; k < slots.size(); k++) {
        Pipeline& P = *slots[k].P;
        // a slot with no room for even one typical event stays unsized (no buffers) until a
        // batch is admitted into it, and is not warmed up: its graph is captured then
        if (b == 0) continue;
        P.ensure_caps(P.estimate(b, (uint32_t)hits_for(b), (uint32_t)pls_for(b)));
        P.ensure_inputs(b, (uint32_t)hits_for(b), (uint32_t)pls_for(b));
        lst_event empty{};
        pack_host_events(P, &empty, 1);
        P.launch(true);
        if (!P.wait(0)) return fail(c, LST_ERR_TIMEOUT, "slot warm-up timed out");
      }
    }
    for (auto& sl : slots) sl.P->byte_cap = budget ? slot_share : 0;
    auto note_bytes = [&] {
      uint64_t t = base;
      for (auto& sl : slots) t += sl.P->dev_bytes;
      uint64_t p = peak.load();
      while (t > p && !peak.compare_exchange_weak(p, t)) {
      }
    };
    note_bytes();
    // Shared state: arrived events not yet taken, and the first error of any worker.
    std::mutex qm;
    // unless the slots share the device, each batch's chain is queued behind the batch
    // launched before it (an event wait on the device: no host round trip between batches)
    std::mutex chain_m;
    cudaEvent_t last_done = nullptr;  // completion event of the last batch launched
    // batches launched and not yet finished (under qm): a slot takes events only when a
    // full batch is waiting or at most one batch is in flight, so under load the batches
    // grow to max_batch instead of launching a few events each while the device is busy
    uint32_t in_flight = 0;
    const bool share = cfg->share_device != 0;
    std::condition_variable qcv;
    std::deque<uint32_t> queue;
    bool closed = false;
    lst_status status = LST_OK;
    std::string err_msg;
    const double t0 = now_s();
    auto set_error = [&](lst_status st, const std::string& m) {
      std::lock_guard<std::mutex> lk(qm);
      if (status == LST_OK) {
        status = st;
        err_msg = m;
      }
      qcv.notify_all();
    };
    // One worker per slot: take what has arrived (up to max_batch events within the memory
    // budget), upload, replay the slot's graph, wait, collect, stamp the latencies.
    auto worker = [&](size_t k) {
      Pipeline& P = *slots[k].P;
      try {
        CK(cudaSetDevice(c->device));
        std::vector<uint32_t> take;
        std::vector<lst_event> batch;
        std::vector<uint32_t> tcn;
        std::vector<lst_result_id> ids;
        for (;;) {
          take.clear();
          batch.clear();
          {
            std::unique_lock<std::mutex> lk(qm);
            qcv.wait(lk, [&] {
              return (!queue.empty() && (queue.size() >= cfg->max_batch || in_flight <= 1 || closed)) ||
                     (queue.empty() && closed) || status != LST_OK;
            });
            if (status != LST_OK || (queue.empty() && closed)) return;
            uint64_t nh = 0, np = 0;
            while (!queue.empty() && take.size() < cfg->max_batch) {
              const lst_event& e = evs[queue.front()];
              if (!fits(P, (uint32_t)take.size() + 1, nh + e.n_hits, np + e.n_pls)) {
                if (take.empty()) {
                  const uint64_t need = P.bytes_after(P.estimate(1, e.n_hits, e.n_pls), 1, e.n_hits, e.n_pls);
                  lk.unlock();
                  char msg[256];
                  snprintf(msg, sizeof msg,
                           "one event alone (%u hits, %u seeds) needs %llu bytes in its slot, more than the slot's "
                           "share of the memory budget (%llu bytes; the slot holds %llu)",
                           e.n_hits, e.n_pls, (unsigned long long)need, (unsigned long long)slot_share,
                           (unsigned long long)P.dev_bytes);
                  return set_error(LST_ERR_BUDGET, msg);
                }
                break;
              }
              take.push_back(queue.front());
              nh += e.n_hits;
              np += e.n_pls;
              queue.pop_front();
            }
          }
          {
            std::lock_guard<std::mutex> lk(qm);
            in_flight++;
          }
          for (uint32_t i : take) batch.push_back(evs[i]);
          pack_host_events(P, batch.data(), (uint32_t)batch.size());
          P.ensure_caps(P.estimate((uint32_t)batch.size(), P.n_hits, P.n_pls));
          note_bytes();
          n_batches++;
          for (uint32_t mt = max_taken.load(); take.size() > mt && !max_taken.compare_exchange_weak(mt, (uint32_t)take.size());) {
          }
          for (int attempt = 0;; attempt++) {
            if (share) {
              P.launch(true);
            } else {
              std::lock_guard<std::mutex> lk(chain_m);
              P.launch(true, nullptr, last_done);
              last_done = P.done;
            }
            if (!P.wait(0)) return set_error(LST_ERR_TIMEOUT, "device did not finish");
            const Hdr& h = *P.h_hdr_out;
            if (h.err & ERR_BAD_INPUT) return set_error(LST_ERR_BAD_INPUT, "bad input in a served event");
            if (h.err & ERR_WAIT) return set_error(LST_ERR_TIMEOUT, "a bounded device-side wait ran out");
            if (!P.grow_after_overflow(h)) {
              P.learn(h);
              break;
            }
            note_bytes();
            if (budget && P.dev_bytes > slot_share)
              return set_error(LST_ERR_BUDGET, "a batch outgrew its slot's share of the memory budget");
            if (attempt > 10) return set_error(LST_ERR_OOM, "object lists kept outgrowing their storage");
            std::lock_guard<std::mutex> lk(c->mu);
            c->reruns++;
          }
          {
            std::lock_guard<std::mutex> lk(qm);
            in_flight--;
          }
          qcv.notify_all();
          tcn.assign(take.size(), 0);
          ids.assign(take.size(), 0);
          collect(c, P, outs ? ids.data() : nullptr, tcn.data());
          const double tdone = now_s() - t0;
          for (size_t q = 0; q < take.size(); q++) {
            const uint32_t e = take[q];
            latency_s[e] = tdone - arrival_s[e];
            if (n_tc) n_tc[e] = tcn[q];
            if (outs) outs[e] = ids[q];
          }
        }
      } catch (const CudaError& e) {
        set_error(LST_ERR_CUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
      } catch (const StatusError& e) {
        set_error(e.s, e.msg);
      } catch (const std::bad_alloc&) {
        set_error(LST_ERR_OOM, "host allocation failed");
      }
    };
    std::vector<std::thread> th;
    for (size_t k = 0; k < slots.size(); k++) th.emplace_back(worker, k);
    // The request loop: release every event at its arrival time.
    for (uint32_t i = 0; i < n;) {
      const double now = now_s() - t0;
      if (arrival_s[i] > now) {
        const double wait = arrival_s[i] - now;
        if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(qm);
        if (status != LST_OK) break;
        while (i < n && arrival_s[i] <= now) queue.push_back(i++);
      }
      qcv.notify_all();
    }
    {
      std::lock_guard<std::mutex> lk(qm);
      closed = true;
    }
    qcv.notify_all();
    for (auto& t : th) t.join();
    if (wall_s) *wall_s = now_s() - t0;
    {
      std::lock_guard<std::mutex> lk(c->mu);
      c->served_batches = n_batches.load();
      c->served_max_batch = max_taken.load();
      c->served_peak_bytes = peak.load();
    }
    if (status != LST_OK) return fail(c, status, err_msg);
    return LST_OK;
  });
}

// ------------------------------------------------------------------ views for lst_static.cu
namespace lst {
bool ctx_views(lst_ctx* c, GeoView* g, MethodConst* m, Launch* l, int* device, bool* have_map) {
  if (!c) return false;
  *g = c->geo.view();
  *m = c->main.C;
  *l = c->main.L;
  l->t5_mlp = c->geo.has_t5_mlp ? &c->geo.t5_mlp : nullptr;
  *device = c->device;
  *have_map = c->geo.have_map;
  return true;
}
void ctx_set_error(lst_ctx* c, const std::string& msg) {
  if (c) c->err = msg;
}
}  // namespace lst
