// Runtime and C ABI of the L.A.Cosmic library (declared in include/lacos.h).
//
// A context owns a fixed set of slots.  A submitted request (one frame or a
// batch) takes a free slot, whose device scratch -- per-frame descriptors,
// per-frame state, two bit-packed mask buffers, three bit-planes and the
// N table per frame, and the tile-queue heads -- is allocated stream-ordered
// and charged against the context's HBM budget.  The request's work is
// queued on the caller's stream:
//   memcpy(descriptors) ; memset(state, heads, M_0) ; ntab_kernel ;
//   { core_kernel<u16>(k) ; core_kernel<f32>(k) ; grow_kernel(k) } for k = 1..max niter ;
//   finalize_kernel ;
// (each core kernel only where the request has frames of its dtype).
//   memcpy(state -> pinned host) ; event.
// Polling queries the event, reads the pinned state and frees the slot.
// Host-to-host requests run on their slot's own stream with the frame's
// upload before and the outputs' download after that sequence.  The kernel
// sequences of host requests whose frame fills the GPU kChainWaves times
// over are chained through one context event (each waits for the previous
// such request's finalize_kernel), so that requests in flight run their
// kernels one after another while the copies of the requests before and
// after overlap them, instead of sharing the SMs, finishing together and
// then downloading back to back.  Smaller frames cannot fill the GPU alone
// and keep running concurrently.
// Iteration control is on the device: an iteration whose predecessor
// flagged nothing returns at once, so the host never waits mid-request.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "lacos_kernels.cuh"

using namespace lacos;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kNtabBytes = 65536 * sizeof(float2);  // {2N, 1/(2N)} per uint16 med5 value
// Histogram of the pair differences of a frame whose gain is estimated: a
// count (u32) and a sum of a + b (u64) per d.
constexpr size_t kGainHistN = ((size_t)kGainBins * sizeof(unsigned) + 255) / 256 * 256;
constexpr size_t kGainHistBytes = kGainHistN + ((size_t)kGainBins * sizeof(unsigned long long) + 255) / 256 * 256;
// Tile-queue heads: one per (core kernel dtype, level) plus the final replace.
constexpr int kHeadLevels = LACOS_MAX_NITER + 1;
constexpr int kHeadCore = 0;  // + dtype * kHeadLevels + level
constexpr int kHeadFinal = 2 * kHeadLevels, kHeads = kHeadFinal + 1;
inline size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

struct FrameReq {
  const void* frame;
  int dtype, ny, nx;
  lacos_params p;
  uint8_t* mask;
  float* clean;
};

// Host buffers of a lacos_submit_host request.
struct HostIO {
  const void* frame;
  uint8_t* mask;
  float* clean;
};

struct Slot {
  bool busy = false;
  unsigned long long ticket = 0;
  void* dscratch = nullptr;  // device scratch
  size_t dcap = 0;
  void* dio = nullptr;       // device copies of a host request's frame, mask and cleaned frame
  size_t iocap = 0;
  void* hpinned = nullptr;   // pinned host staging (descriptors in, states out)
  size_t hcap = 0;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  int nframes = 0;
  lacos_result* per_frame = nullptr;  // caller's array for batch results
  // CUDA graph of the last batch (replayed when the same batch comes back).
  cudaGraphExec_t gexec = nullptr;
  std::vector<FrameReq> graph_key;
  cudaStream_t cap_stream = nullptr;  // capture stream (the caller's may be uncapturable)
  cudaStream_t own_stream = nullptr;  // the slot's own stream (lacos_submit_async)
  // Profiling events (see enqueue).
  std::vector<cudaEvent_t> prof_ev;
  int prof_n = -1;  // levels recorded for the request in flight (-1: none)
  std::vector<long long> npix;
  std::vector<float> gain_in;  // per frame: the supplied gain (0: estimated)
};

bool same_batch(const std::vector<FrameReq>& a, const std::vector<FrameReq>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i) {
    if (a[i].frame != b[i].frame || a[i].dtype != b[i].dtype || a[i].ny != b[i].ny ||
        a[i].nx != b[i].nx || a[i].mask != b[i].mask || a[i].clean != b[i].clean ||
        std::memcmp(&a[i].p, &b[i].p, sizeof(lacos_params)) != 0)
      return false;
  }
  return true;
}

int wpr_of(int nx) { return (nx + 31) / 32; }
size_t maskbuf_bytes(int ny, int nx) { return align_up((size_t)ny * wpr_of(nx) * sizeof(uint32_t)); }
// Per-tile level marks of the core kernel: two ping-pong bytes and a sticky one per
// tile, sized for the smallest core tile (32 x 32) so that every variant fits.
size_t tflag_bytes(int ny, int nx) {
  return align_up(3 * (size_t)((nx + G32x32::TW - 1) / G32x32::TW) * (size_t)((ny + G32x32::TH - 1) / G32x32::TH));
}

struct Layout {
  size_t heads, descs, states, masks, total;
  std::vector<size_t> mask_off;
};

Layout layout_for(const std::vector<FrameReq>& fr) {
  Layout L;
  const size_t n = fr.size();
  L.heads = 0;
  L.descs = align_up(sizeof(unsigned) * kHeads);
  L.states = L.descs + align_up(sizeof(FrameDesc) * n);
  L.masks = L.states + align_up(sizeof(FrameState) * n);
  size_t off = L.masks;
  for (const auto& f : fr) {
    L.mask_off.push_back(off);
    // M 0/1, sig/lo/cand, N table, tile marks, with satgrow the grown saturated
    // set, and with an estimated gain the histogram of pair differences
    off += (f.p.satgrow ? 6 : 5) * maskbuf_bytes(f.ny, f.nx) + kNtabBytes + tflag_bytes(f.ny, f.nx) +
           (f.p.gain == 0.0f ? kGainHistBytes : 0);
  }
  L.total = off;
  return L;
}

}  // namespace

// Core-kernel variants: tile geometry (shape, threads per CTA) and the
// resident CTAs per SM its register allocation is bounded for.  0..3 are the
// 32 x 64 tiles at 1..4 CTAs per SM; the others trade more shared memory per
// CTA (and fewer CTAs per SM) for less halo recomputation per pixel.
using CoreFn = void (*)(const FrameDesc*, int, unsigned, unsigned, int, unsigned*);
struct CoreVariant {
  int th, tw, nt, minb;
  CoreFn fn[2];    // by frame dtype (LACOS_F32, LACOS_U16)
  size_t smem[2];  // dynamic shared memory per CTA, by frame dtype
};
template <class G, int MINB>
constexpr CoreVariant make_variant() {
  return {G::TH, G::TW, G::NT, MINB, {core_kernel<G, MINB, float>, core_kernel<G, MINB, uint16_t>},
          {kCoreSmemBytes<G, float>, kCoreSmemBytes<G, uint16_t>}};
}
static const CoreVariant kCoreVariants[LACOS_CORE_VARIANTS] = {
    make_variant<G32x64, 1>(), make_variant<G32x64, 2>(), make_variant<G32x64, 3>(), make_variant<G32x64, 4>(),
    make_variant<G64x64, 1>(), make_variant<G64x64, 2>(), make_variant<G32x128, 1>(), make_variant<G32x128, 2>(),
    make_variant<G32x32, 5>(), make_variant<G32x32, 6>()};
constexpr int kDefaultCoreVariant = 3;

struct lacos_ctx {
  int device = 0;
  size_t budget = 0;
  size_t charged = 0;
  std::vector<Slot> slots;
  std::mutex mu;
  unsigned long long next_ticket = 1;
  std::atomic<int> last_cuda{0};
  int num_sms = 0;
  int core_variant = kDefaultCoreVariant;  // index into kCoreVariants
  int blocks_per_sm_core_v[2][LACOS_CORE_VARIANTS] = {};  // resident CTAs by dtype and variant
  int blocks_per_sm_final[2] = {1, 1};  // resident finalize CTAs: [small, big tiles]
  bool profiling = false;
  lacos_profile last_prof{};
  cudaEvent_t host_chain = nullptr;     // end of the last host request's kernels
};

// A host request is chained when its tiles number at least kChainWaves
// times the resident core CTAs.
constexpr unsigned kChainWaves = 8;


static int cuda_fail(lacos_ctx* c, cudaError_t e) {
  if (c) c->last_cuda = (int)e;
  return LACOS_ECUDA;
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_); \
  } while (0)

static bool params_valid(const lacos_params* p) {
  if (!p) return false;
  const float v[6] = {p->gain, p->readnoise, p->satlevel, p->sigclip, p->sigfrac, p->objlim};
  for (float x : v)
    if (!std::isfinite(x)) return false;
  if (!(p->gain >= 0.0f) || !(p->readnoise >= 0.0f) || !(p->sigclip > 0.0f) ||
      !(p->sigfrac > 0.0f) || !(p->objlim > 0.0f))
    return false;
  if (p->niter < 0 || p->niter > LACOS_MAX_NITER) return false;
  if (p->fine_norm != 0 && p->fine_norm != 1) return false;
  if (p->satgrow < 0 || p->satgrow > 4) return false;
  if (p->sepmed != 0 && p->sepmed != 1) return false;
  return true;
}

static bool frame_valid(const FrameReq& f) {
  if (!f.frame || !f.mask || !f.clean) return false;
  if (f.dtype != LACOS_F32 && f.dtype != LACOS_U16) return false;
  if (f.ny < 1 || f.nx < 1) return false;
  if ((long long)f.ny * (long long)f.nx >= (1LL << 31)) return false;
  if (f.p.gain == 0.0f && f.dtype != LACOS_U16) return false;  // estimated gain: integer frames only
  return params_valid(&f.p);
}

// Frees idle slots' scratch until `need` more bytes fit the budget.
static void evict_idle(lacos_ctx* c, size_t need, cudaStream_t s) {
  for (auto& sl : c->slots) {
    if (c->charged + need <= c->budget) return;
    if (!sl.busy && sl.dscratch) {
      cudaFreeAsync(sl.dscratch, s);
      c->charged -= sl.dcap;
      sl.dscratch = nullptr;
      sl.dcap = 0;
      if (sl.gexec) { cudaGraphExecDestroy(sl.gexec); sl.gexec = nullptr; sl.graph_key.clear(); }
    }
    if (!sl.busy && sl.dio && c->charged + need > c->budget) {
      cudaFreeAsync(sl.dio, s);
      c->charged -= sl.iocap;
      sl.dio = nullptr;
      sl.iocap = 0;
    }
  }
}

// Gain estimation (frames with gain 0) at level k: the histogram of pair
// differences (four CTAs per SM per frame; the kernel is bounded to 64
// registers for four resident CTAs), the clipping rounds on it (one block per
// frame), then the N table where the gain changed.
static void launch_gain_level(const FrameDesc* ddesc, int nf, int k, int num_sms, cudaStream_t s) {
  gain_hist_kernel<<<dim3((unsigned)(4 * num_sms), (unsigned)nf), kBlock, 0, s>>>(ddesc, nf, k);
  gain_fold_kernel<<<(unsigned)nf, kFoldThreads, 0, s>>>(ddesc, nf, k);
  ntab_level_kernel<<<dim3(256, (unsigned)nf), 256, 0, s>>>(ddesc, nf, k);
}

// Growth and finalize shapes of a request: the larger blocks from 8 Mpx of
// frames on (a 61-Mpx frame takes 12% less time per growth level and 18%
// less in finalize with them); below that they would leave the GPU with too
// few blocks (a 512 x 512 frame was 7% slower per request).
constexpr unsigned long long kBigShapePx = 8ull << 20;
struct PassShapes {
  bool big;
  int fth, ftw, gh, gw;
};
static PassShapes pass_shapes(unsigned long long px) {
  const bool big = px >= kBigShapePx;
  return big ? PassShapes{true, FGBig::TH, FGBig::TW, GrowBig::H, GrowBig::W}
             : PassShapes{false, FGSmall::TH, FGSmall::TW, GrowSmall::H, GrowSmall::W};
}
static void launch_grow(bool big, unsigned nblk, const FrameDesc* ddesc, int nf, int k, cudaStream_t s) {
  if (big)
    grow_kernel<GrowBig><<<nblk, kBlock, 0, s>>>(ddesc, nf, nblk, k);
  else
    grow_kernel<GrowSmall><<<nblk, kBlock, 0, s>>>(ddesc, nf, nblk, k);
}
static void launch_finalize(bool big, unsigned grid, const FrameDesc* ddesc, int nf, unsigned total,
                            unsigned* head, cudaStream_t s) {
  if (big)
    finalize_kernel<FGBig><<<grid, kBlock, 0, s>>>(ddesc, nf, total, head);
  else
    finalize_kernel<FGSmall><<<grid, kBlock, 0, s>>>(ddesc, nf, total, head);
}

// `chain`, when given, is waited on before the first kernel (after the
// descriptor copy and memsets, which touch only this slot's scratch) and
// recorded after finalize_kernel (before the state copy, which may queue
// behind another request's download).
static int enqueue(lacos_ctx* c, Slot& sl, const std::vector<FrameReq>& fr, const Layout& L,
                   cudaStream_t s, bool prof, cudaEvent_t chain = nullptr) {
  char* d = (char*)sl.dscratch;
  const int cv = c->core_variant;
  const CoreVariant& V = kCoreVariants[cv];
  unsigned* heads = (unsigned*)(d + L.heads);
  FrameDesc* ddesc = (FrameDesc*)(d + L.descs);
  FrameState* dstate = (FrameState*)(d + L.states);
  // Host descriptors in the pinned buffer (states come back after them).
  FrameDesc* hdesc = (FrameDesc*)sl.hpinned;
  unsigned total = 0, total_fin = 0;
  unsigned long long total_words = 0;
  unsigned total_gblk = 0;
  int max_niter = 0;
  // Descriptor order: uint16 frames first, so that each dtype's tiles form
  // one contiguous item range for its core kernel.  Each descriptor keeps
  // its frame's own state and scratch (request order).
  std::vector<size_t> order;
  order.reserve(fr.size());
  for (int dt : {1, 0})
    for (size_t i = 0; i < fr.size(); ++i)
      if (fr[i].dtype == dt) order.push_back(i);
  unsigned tiles_u16 = 0;
  bool any_est = false;
  unsigned long long req_px = 0;
  for (const FrameReq& f : fr) req_px += (unsigned long long)f.ny * (unsigned long long)f.nx;
  const PassShapes ps = pass_shapes(req_px);
  for (size_t j = 0; j < fr.size(); ++j) {
    const size_t i = order[j];
    const FrameReq& f = fr[i];
    FrameDesc& h = hdesc[j];
    std::memset(&h, 0, sizeof(h));
    h.x0 = f.frame;
    h.dtype = f.dtype;
    h.ny = f.ny;
    h.nx = f.nx;
    h.wpr = wpr_of(f.nx);
    const size_t mb = maskbuf_bytes(f.ny, f.nx);
    h.mbuf0 = (uint32_t*)(d + L.mask_off[i]);
    h.mbuf1 = (uint32_t*)(d + L.mask_off[i] + mb);
    h.p_sig = (uint32_t*)(d + L.mask_off[i] + 2 * mb);
    h.p_lo = (uint32_t*)(d + L.mask_off[i] + 3 * mb);
    h.p_cand = (uint32_t*)(d + L.mask_off[i] + 4 * mb);
    h.ntab = (float2*)(d + L.mask_off[i] + 5 * mb);
    h.tflags = (uint8_t*)(d + L.mask_off[i] + 5 * mb + kNtabBytes);
    char* after = d + L.mask_off[i] + 5 * mb + kNtabBytes + tflag_bytes(f.ny, f.nx);
    h.p_sat = f.p.satgrow ? (uint32_t*)after : nullptr;
    if (f.p.satgrow) after += mb;
    h.ghist_n = f.p.gain == 0.0f ? (unsigned*)after : nullptr;
    h.ghist_a = f.p.gain == 0.0f ? (unsigned long long*)(after + kGainHistN) : nullptr;
    h.mask_out = f.mask;
    h.clean_out = f.clean;
    h.st = dstate + i;
    h.gain = f.p.gain;
    h.gain_est = f.p.gain == 0.0f;
    any_est = any_est || h.gain_est;
    h.rn = f.p.readnoise;
    volatile float rn = f.p.readnoise;
    volatile float rn2 = rn * rn;  // float product, as the float32 definition
    h.rn2 = rn2;
    h.satlevel = f.p.satlevel;
    h.sigclip = f.p.sigclip;
    volatile float lo = f.p.sigfrac * f.p.sigclip;
    h.lo = lo;
    h.thr_min = std::min(h.lo, h.sigclip);
    h.objlim = f.p.objlim;
    h.niter = f.p.niter;
    h.fnorm = f.p.fine_norm;
    h.satgrow = f.p.satgrow;
    h.sepmed = f.p.sepmed;
    h.th = V.th;
    h.tw = V.tw;
    h.tiles_x = (f.nx + V.tw - 1) / V.tw;
    const unsigned tiles = (unsigned)h.tiles_x * (unsigned)((f.ny + V.th - 1) / V.th);
    h.tile_begin = total;
    total += tiles;
    h.tile_end = total;
    if (f.dtype == LACOS_U16) tiles_u16 = total;
    h.ftiles_x = (f.nx + ps.ftw - 1) / ps.ftw;
    h.fin_begin = total_fin;
    total_fin += (unsigned)h.ftiles_x * (unsigned)((f.ny + ps.fth - 1) / ps.fth);
    h.fin_end = total_fin;
    h.word_begin = total_words;
    total_words += (unsigned long long)f.ny * h.wpr;
    h.gblk_x = (unsigned)((h.wpr + ps.gw - 1) / ps.gw);
    h.gblk_begin = total_gblk;
    total_gblk += h.gblk_x * (unsigned)((f.ny + ps.gh - 1) / ps.gh);
    max_niter = std::max(max_niter, f.p.niter);
  }
  CK(cudaMemcpyAsync(ddesc, hdesc, sizeof(FrameDesc) * fr.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(heads, 0, sizeof(unsigned) * kHeads, s));
  CK(cudaMemsetAsync(dstate, 0, sizeof(FrameState) * fr.size(), s));
  for (size_t j = 0; j < fr.size(); ++j) {
    const size_t i = order[j];
    const size_t mb = maskbuf_bytes(fr[i].ny, fr[i].nx);
    CK(cudaMemsetAsync(d + L.mask_off[i], 0, mb, s));  // M_0
    CK(cudaMemsetAsync(d + L.mask_off[i] + 5 * mb + kNtabBytes, 0, tflag_bytes(fr[i].ny, fr[i].nx), s));
    if (hdesc[j].ghist_n) CK(cudaMemsetAsync(hdesc[j].ghist_n, 0, kGainHistBytes, s));
  }
  const int nf = (int)fr.size();
  // Core launches: [dtype] -> item range and grid.
  const unsigned rng[2][2] = {{tiles_u16, total}, {0, tiles_u16}};
  unsigned gdt[2];
  for (int dt = 0; dt < 2; ++dt)
    gdt[dt] = std::min<unsigned>(rng[dt][1] - rng[dt][0],
                                 (unsigned)(c->num_sms * c->blocks_per_sm_core_v[dt][cv]));
  const unsigned gfi = std::min<unsigned>(total_fin, (unsigned)(c->num_sms * c->blocks_per_sm_final[ps.big]));
  // Profile events: [0] start, level k: [2k-1] after core, [2k] after grow,
  // [2n+1] after finalize.
  const int nev = 2 * max_niter + 2;
  if (chain) CK(cudaStreamWaitEvent(s, chain, 0));
  if (prof) {
    while ((int)sl.prof_ev.size() < nev) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      sl.prof_ev.push_back(e);
    }
    CK(cudaEventRecord(sl.prof_ev[0], s));
  }
  auto mark = [&](int i) -> int {
    if (prof) CK(cudaEventRecord(sl.prof_ev[i], s));
    return LACOS_OK;
  };
  ntab_kernel<<<dim3(256, nf), 256, 0, s>>>(ddesc, nf);
  for (size_t j = 0; j < fr.size(); ++j) {  // the grown saturated sets (C16)
    const FrameReq& f = fr[order[j]];
    if (!f.p.satgrow) continue;
    const unsigned nw = (unsigned)((size_t)f.ny * wpr_of(f.nx));
    satseed_kernel<<<(nw + 255) / 256, 256, 0, s>>>(ddesc, (int)j, nw);
    satgrow_kernel<<<(nw + 255) / 256, 256, 0, s>>>(ddesc, (int)j, nw);
  }
  CK(cudaGetLastError());
  for (int k = 1; k <= max_niter; ++k) {
    if (any_est) {
      launch_gain_level(ddesc, nf, k, c->num_sms, s);
      CK(cudaGetLastError());
    }
    for (int dt : {1, 0}) {
      if (!gdt[dt]) continue;
      V.fn[dt]<<<gdt[dt], V.nt, V.smem[dt], s>>>(ddesc, nf, rng[dt][0], rng[dt][1], k,
                                                  heads + kHeadCore + dt * kHeadLevels + k);
      CK(cudaGetLastError());
    }
    if (int rc = mark(2 * k - 1)) return rc;
    launch_grow(ps.big, total_gblk, ddesc, nf, k, s);
    CK(cudaGetLastError());
    if (int rc = mark(2 * k)) return rc;
  }
  launch_finalize(ps.big, gfi, ddesc, nf, total_fin, heads + kHeadFinal, s);
  CK(cudaGetLastError());
  if (int rc = mark(2 * max_niter + 1)) return rc;
  if (chain) CK(cudaEventRecord(chain, s));
  sl.prof_n = prof ? max_niter : -1;
  FrameState* hstate = (FrameState*)((char*)sl.hpinned + align_up(sizeof(FrameDesc) * fr.size()));
  CK(cudaMemcpyAsync(hstate, dstate, sizeof(FrameState) * fr.size(), cudaMemcpyDeviceToHost, s));
  return LACOS_OK;
}

static int submit_impl(lacos_ctx* c, const std::vector<FrameReq>& fr_in, cudaStream_t s,
                       int reuse_graph, lacos_result* per_frame, unsigned long long* ticket,
                       bool own_stream = false, const HostIO* hio = nullptr) {
  if (!c || !ticket || fr_in.empty()) return LACOS_EINVAL;
  for (const auto& f : fr_in)
    if (!frame_valid(f)) return LACOS_EINVAL;
  std::vector<FrameReq> fr = fr_in;
  const Layout L = layout_for(fr);
  // A host request (one frame) also needs device copies of its frame and outputs.
  const size_t npx = hio ? (size_t)fr[0].ny * fr[0].nx : 0;
  const size_t io_frame = align_up(npx * (fr[0].dtype == LACOS_U16 ? 2 : 4)), io_mask = align_up(npx);
  const size_t io_need = hio ? io_frame + io_mask + align_up(npx * sizeof(float)) : 0;
  const size_t hneed = align_up(sizeof(FrameDesc) * fr.size()) + sizeof(FrameState) * fr.size();
  std::lock_guard<std::mutex> lk(c->mu);
  if (L.total + io_need > c->budget) return LACOS_ENOMEM;
  CK(cudaSetDevice(c->device));
  // Pick a free slot, preferring one whose scratch is already large enough.
  Slot* sl = nullptr;
  for (auto& x : c->slots)
    if (!x.busy && x.dcap >= L.total) { sl = &x; break; }
  if (!sl)
    for (auto& x : c->slots)
      if (!x.busy) { sl = &x; break; }
  if (!sl) return LACOS_EAGAIN;
  if (own_stream) {
    if (!sl->own_stream) CK(cudaStreamCreateWithFlags(&sl->own_stream, cudaStreamNonBlocking));
    s = sl->own_stream;
  }
  if (sl->dcap < L.total) {
    if (sl->dscratch) {
      CK(cudaFreeAsync(sl->dscratch, s));
      c->charged -= sl->dcap;
      sl->dscratch = nullptr;
      sl->dcap = 0;
      if (sl->gexec) { cudaGraphExecDestroy(sl->gexec); sl->gexec = nullptr; sl->graph_key.clear(); }
    }
    evict_idle(c, L.total, s);
    if (c->charged + L.total > c->budget) return LACOS_EAGAIN;
    CK(cudaMallocAsync(&sl->dscratch, L.total, s));
    sl->dcap = L.total;
    c->charged += L.total;
  }
  if (sl->iocap < io_need) {
    if (sl->dio) {
      CK(cudaFreeAsync(sl->dio, s));
      c->charged -= sl->iocap;
      sl->dio = nullptr;
      sl->iocap = 0;
    }
    evict_idle(c, io_need, s);
    if (c->charged + io_need > c->budget) return LACOS_EAGAIN;
    CK(cudaMallocAsync(&sl->dio, io_need, s));
    sl->iocap = io_need;
    c->charged += io_need;
  }
  if (hio) {  // the request reads and writes the slot's device copies
    char* io = (char*)sl->dio;
    fr[0].frame = io;
    fr[0].mask = (uint8_t*)(io + io_frame);
    fr[0].clean = (float*)(io + io_frame + io_mask);
  }
  if (sl->hcap < hneed) {
    if (sl->hpinned) { CK(cudaStreamSynchronize(s)); cudaFreeHost(sl->hpinned); }
    if (sl->gexec) { cudaGraphExecDestroy(sl->gexec); sl->gexec = nullptr; sl->graph_key.clear(); }
    sl->hpinned = nullptr;
    sl->hcap = 0;
    CK(cudaMallocHost(&sl->hpinned, hneed));
    sl->hcap = hneed;
  }
  if (hio && !c->host_chain) CK(cudaEventCreateWithFlags(&c->host_chain, cudaEventDisableTiming));
  if (!sl->ev_start) CK(cudaEventCreate(&sl->ev_start));
  if (!sl->ev_done) CK(cudaEventCreate(&sl->ev_done));
  CK(cudaEventRecord(sl->ev_start, s));
  int rc;
  if (reuse_graph && sl->gexec && same_batch(sl->graph_key, fr)) {
    CK(cudaGraphLaunch(sl->gexec, s));
    sl->prof_n = -1;
    rc = LACOS_OK;
  } else if (reuse_graph) {
    // Capture on the slot's own stream, then launch the graph on the caller's.
    if (!sl->cap_stream) CK(cudaStreamCreateWithFlags(&sl->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(sl->cap_stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue(c, *sl, fr, L, sl->cap_stream, false);
    cudaError_t e = cudaStreamEndCapture(sl->cap_stream, &g);
    if (rc != LACOS_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(c, e);
    if (sl->gexec) cudaGraphExecDestroy(sl->gexec);
    sl->gexec = nullptr;
    e = cudaGraphInstantiate(&sl->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e);
    sl->graph_key = fr;
    sl->prof_n = -1;
    CK(cudaGraphLaunch(sl->gexec, s));
  } else {
    if (hio)
      CK(cudaMemcpyAsync((void*)fr[0].frame, hio->frame, npx * (fr[0].dtype == LACOS_U16 ? 2 : 4),
                         cudaMemcpyHostToDevice, s));
    bool chain = false;
    if (hio) {
      const CoreVariant& V = kCoreVariants[c->core_variant];
      const unsigned tiles = (unsigned)((fr[0].ny + V.th - 1) / V.th) * (unsigned)((fr[0].nx + V.tw - 1) / V.tw);
      const unsigned resident = (unsigned)c->num_sms * (unsigned)c->blocks_per_sm_core_v[fr[0].dtype][c->core_variant];
      chain = tiles >= kChainWaves * resident;
    }
    rc = enqueue(c, *sl, fr, L, s, c->profiling, chain ? c->host_chain : nullptr);
    if (rc != LACOS_OK) return rc;
    if (hio) {
      CK(cudaMemcpyAsync(hio->mask, fr[0].mask, npx, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hio->clean, fr[0].clean, npx * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
  }
  CK(cudaEventRecord(sl->ev_done, s));
  sl->busy = true;
  sl->nframes = (int)fr.size();
  sl->npix.resize(fr.size());
  sl->gain_in.resize(fr.size());
  for (size_t i = 0; i < fr.size(); ++i) {
    sl->npix[i] = (long long)fr[i].ny * fr[i].nx;
    sl->gain_in[i] = fr[i].p.gain;
  }
  sl->per_frame = per_frame;
  sl->ticket = c->next_ticket++;
  *ticket = sl->ticket;
  return LACOS_OK;
}

static int finish(lacos_ctx* c, Slot& sl, lacos_result* res) {
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, sl.ev_start, sl.ev_done);
  const FrameState* hs = (const FrameState*)((char*)sl.hpinned + align_up(sizeof(FrameDesc) * sl.nframes));
  lacos_result agg{LACOS_OK, 0, 0, (double)ms, 0.0f};
  if (sl.prof_n >= 0) {
    lacos_profile& P = c->last_prof;
    std::memset(&P, 0, sizeof(P));
    P.n_levels = sl.prof_n;
    const auto& E = sl.prof_ev;
    for (int k = 1; k <= sl.prof_n; ++k) {
      cudaEventElapsedTime(&P.core_ms[k - 1], E[2 * k - 2], E[2 * k - 1]);
      cudaEventElapsedTime(&P.grow_ms[k - 1], E[2 * k - 1], E[2 * k]);
    }
    cudaEventElapsedTime(&P.final_ms, E[2 * sl.prof_n], E[2 * sl.prof_n + 1]);
    for (int i = 0; i < sl.nframes; ++i) {
      P.px_iterations += sl.npix[i] * hs[i].iters_run;
      P.n_sprime += (long long)hs[i].n_sprime;
      P.n_fine += (long long)hs[i].n_fine;
      P.n_replace += (long long)hs[i].n_replace;
      P.n_replace_wide += (long long)hs[i].n_replace_wide;
      P.px_core += (long long)hs[i].px_core;
      P.n_sprime_net += (long long)hs[i].n_sprime_net;
      P.n_fine_net += (long long)hs[i].n_fine_net;
    }
  }
  for (int i = 0; i < sl.nframes; ++i) {
    lacos_result r{LACOS_OK, hs[i].iters_run, (long long)hs[i].flagged, (double)ms, 0.0f};
    r.gain = sl.gain_in[i] > 0.0f ? sl.gain_in[i] : hs[i].gain;
    if (hs[i].err & ERR_NONFINITE) r.status = LACOS_ENONFINITE;
    else if (hs[i].err & ERR_TIMEOUT) r.status = LACOS_ETIMEOUT;
    else if (hs[i].err & ERR_NOGAIN) r.status = LACOS_ENOGAIN;
    if (sl.per_frame) sl.per_frame[i] = r;
    if (agg.status == LACOS_OK) agg.status = r.status;
    agg.iters_run = std::max(agg.iters_run, r.iters_run);
    agg.n_flagged += r.n_flagged;
    agg.gain = sl.nframes == 1 ? r.gain : 0.0f;
  }
  if (res) *res = agg;
  sl.busy = false;
  sl.per_frame = nullptr;
  return LACOS_OK;
}

extern "C" {

const char* lacos_version(void) { return "lacos-gb300 0.4 (sm_103a)"; }

int lacos_selftest_division(float gain, float readnoise, unsigned long long* mismatches) {
  if (!mismatches || !(gain > 0.0f) || !(readnoise >= 0.0f) || !std::isfinite(gain) || !std::isfinite(readnoise))
    return LACOS_EINVAL;
  FrameDesc f;
  std::memset(&f, 0, sizeof(f));
  f.dtype = LACOS_U16;
  f.gain = gain;
  volatile float rn = readnoise;
  volatile float rn2 = rn * rn;  // as a request forms it
  f.rn2 = rn2;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return LACOS_ECUDA;
  cudaError_t e = cudaMemset(d, 0, sizeof(*d));
  if (e == cudaSuccess) {
    selftest_division_kernel<<<65536, 256>>>(f, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(mismatches, d, sizeof(*d), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? LACOS_OK : LACOS_ECUDA;
}

size_t lacos_scratch_bytes(int ny, int nx) { return lacos_request_bytes(ny, nx, nullptr); }

size_t lacos_request_bytes(int ny, int nx, const lacos_params* p) {
  if (ny < 1 || nx < 1) return 0;
  std::vector<FrameReq> fr(1);
  std::memset(&fr[0], 0, sizeof(FrameReq));
  fr[0].ny = ny;
  fr[0].nx = nx;
  fr[0].p.gain = 1.0f;  // defaults: a supplied gain, no saturated-star protection
  if (p) fr[0].p = *p;
  return layout_for(fr).total;
}

int lacos_create(lacos_ctx** out, int device, size_t hbm_budget_bytes, int max_slots) {
  if (!out || device < 0 || max_slots < 0) return LACOS_EINVAL;
  *out = nullptr;
  lacos_ctx* c = new lacos_ctx();
  c->device = device;
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t(8) << 30);
  c->slots.resize(max_slots ? max_slots : 64);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  for (int dt = 0; dt < 2; ++dt)
    for (int v = 0; v < LACOS_CORE_VARIANTS && e == cudaSuccess; ++v) {
      const CoreVariant& V = kCoreVariants[v];
      e = cudaFuncSetAttribute(V.fn[dt], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V.smem[dt]);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->blocks_per_sm_core_v[dt][v], V.fn[dt], V.nt,
                                                          V.smem[dt]);
      c->blocks_per_sm_core_v[dt][v] = std::max(1, c->blocks_per_sm_core_v[dt][v]);
    }
  if (const char* env = std::getenv("LACOS_CORE_VARIANT")) {
    const int v = std::atoi(env);
    if (v >= 0 && v < LACOS_CORE_VARIANTS) c->core_variant = v;
  }
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->blocks_per_sm_final[0], finalize_kernel<FGSmall>,
                                                      kBlock, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->blocks_per_sm_final[1], finalize_kernel<FGBig>,
                                                      kBlock, 0);
  if (e != cudaSuccess) {
    delete c;
    return LACOS_ECUDA;
  }
  for (int& b : c->blocks_per_sm_final) b = std::max(1, b);
  *out = c;
  return LACOS_OK;
}

int lacos_submit(lacos_ctx* c, const void* d_frame, lacos_dtype dt, int ny, int nx,
                 const lacos_params* p, uint8_t* d_mask, float* d_clean, lacos_stream stream,
                 unsigned long long* ticket) {
  if (!p) return LACOS_EINVAL;
  std::vector<FrameReq> fr{{d_frame, (int)dt, ny, nx, *p, d_mask, d_clean}};
  return submit_impl(c, fr, (cudaStream_t)stream, 0, nullptr, ticket);
}

int lacos_submit_batch(lacos_ctx* c, int n, const void* const* d_frames, const int* dtypes,
                       const int* ny, const int* nx, const lacos_params* params,
                       uint8_t* const* d_masks, float* const* d_cleans, lacos_stream stream,
                       int reuse_graph, lacos_result* per_frame, unsigned long long* ticket) {
  // Per-frame kernels put the frames on the grid's y dimension (at most 65535).
  if (n < 1 || n > 65535 || !d_frames || !dtypes || !ny || !nx || !params || !d_masks || !d_cleans)
    return LACOS_EINVAL;
  std::vector<FrameReq> fr((size_t)n);
  for (int i = 0; i < n; ++i)
    fr[i] = {d_frames[i], dtypes[i], ny[i], nx[i], params[i], d_masks[i], d_cleans[i]};
  return submit_impl(c, fr, (cudaStream_t)stream, reuse_graph, per_frame, ticket);
}

int lacos_submit_async(lacos_ctx* c, const void* d_frame, lacos_dtype dt, int ny, int nx,
                       const lacos_params* p, uint8_t* d_mask, float* d_clean,
                       unsigned long long* ticket) {
  if (!p) return LACOS_EINVAL;
  std::vector<FrameReq> fr{{d_frame, (int)dt, ny, nx, *p, d_mask, d_clean}};
  return submit_impl(c, fr, nullptr, 0, nullptr, ticket, true);
}

int lacos_submit_host(lacos_ctx* c, const void* h_frame, lacos_dtype dt, int ny, int nx,
                      const lacos_params* p, uint8_t* h_mask, float* h_clean,
                      unsigned long long* ticket) {
  if (!p || !h_frame || !h_mask || !h_clean) return LACOS_EINVAL;
  // Placeholder device pointers pass validation; the slot's copies replace them.
  std::vector<FrameReq> fr{{h_frame, (int)dt, ny, nx, *p, h_mask, h_clean}};
  const HostIO hio{h_frame, h_mask, h_clean};
  return submit_impl(c, fr, nullptr, 0, nullptr, ticket, true, &hio);
}

int lacos_set_core_variant(lacos_ctx* c, int variant) {
  if (!c || variant < 0 || variant >= LACOS_CORE_VARIANTS) return LACOS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->core_variant = variant;
  return LACOS_OK;
}

int lacos_get_core_variant(lacos_ctx* c, int* variant) {
  if (!c || !variant) return LACOS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  *variant = c->core_variant;
  return LACOS_OK;
}

int lacos_autotune(lacos_ctx* c, const void* d_frame, lacos_dtype dt, int ny, int nx,
                   const lacos_params* p, uint8_t* d_mask, float* d_clean, lacos_stream stream,
                   int reps, int* best_variant, float* variant_ms) {
  if (!c || !p || reps < 1) return LACOS_EINVAL;
  int best = -1;
  float best_ms = 0.0f;
  for (int v = 0; v < LACOS_CORE_VARIANTS; ++v) {
    int rc = lacos_set_core_variant(c, v);
    if (rc) return rc;
    double sum = 0.0;
    for (int r = 0; r <= reps; ++r) {  // the first run warms up
      unsigned long long t = 0;
      lacos_result res{};
      rc = lacos_submit(c, d_frame, dt, ny, nx, p, d_mask, d_clean, stream, &t);
      if (rc) return rc;
      rc = lacos_wait(c, t, &res);
      if (rc) return rc;
      if (r > 0) sum += res.latency_ms;
    }
    const float ms = (float)(sum / reps);
    if (variant_ms) variant_ms[v] = ms;
    if (best < 0 || ms < best_ms) { best = v; best_ms = ms; }
  }
  if (best_variant) *best_variant = best;
  return lacos_set_core_variant(c, best);
}

int lacos_poll(lacos_ctx* c, unsigned long long ticket, lacos_result* res) {
  if (!c) return LACOS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  for (auto& sl : c->slots) {
    if (!sl.busy || sl.ticket != ticket) continue;
    cudaError_t e = cudaEventQuery(sl.ev_done);
    if (e == cudaErrorNotReady) return LACOS_PENDING;
    if (e != cudaSuccess) return cuda_fail(c, e);
    return finish(c, sl, res);
  }
  return LACOS_EUNKNOWN_TICKET;
}

int lacos_wait(lacos_ctx* c, unsigned long long ticket, lacos_result* res) {
  if (!c) return LACOS_EINVAL;
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    for (auto& sl : c->slots)
      if (sl.busy && sl.ticket == ticket) ev = sl.ev_done;
  }
  if (!ev) return LACOS_EUNKNOWN_TICKET;
  cudaError_t e = cudaEventSynchronize(ev);
  if (e != cudaSuccess) return cuda_fail(c, e);
  return lacos_poll(c, ticket, res);
}

int lacos_last_cuda_error(lacos_ctx* c) { return c ? c->last_cuda.load() : 0; }

int lacos_set_profiling(lacos_ctx* c, int on) {
  if (!c) return LACOS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  c->profiling = on != 0;
  return LACOS_OK;
}

int lacos_last_profile(lacos_ctx* c, lacos_profile* out) {
  if (!c || !out) return LACOS_EINVAL;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->last_prof;
  return LACOS_OK;
}

int lacos_destroy(lacos_ctx* c) {
  if (!c) return LACOS_EINVAL;
  cudaSetDevice(c->device);
  int rc = LACOS_OK;
  for (auto& sl : c->slots) {
    if (sl.ev_done && cudaEventSynchronize(sl.ev_done) != cudaSuccess) rc = LACOS_ECUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) rc = LACOS_ECUDA;
  for (auto& sl : c->slots) {
    if (sl.gexec) cudaGraphExecDestroy(sl.gexec);
    if (sl.dscratch) cudaFree(sl.dscratch);
    if (sl.dio) cudaFree(sl.dio);
    if (sl.hpinned) cudaFreeHost(sl.hpinned);
    if (sl.ev_start) cudaEventDestroy(sl.ev_start);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    for (cudaEvent_t e : sl.prof_ev) cudaEventDestroy(e);
    if (sl.cap_stream) cudaStreamDestroy(sl.cap_stream);
    if (sl.own_stream) cudaStreamDestroy(sl.own_stream);
  }
  if (c->host_chain) cudaEventDestroy(c->host_chain);
  delete c;
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Entry point without device allocation.
//
// Some callers cannot allocate device memory while they run: an acquisition
// pipeline that has planned every byte of the GPU up front and forbids
// cudaMalloc after start-up (an allocation can synchronise the device and
// would break its memory plan), or a host application whose own allocator
// owns the device and lets plugins use only what they bring.  For them,
// lacos_run_static does the whole detect-and-clean of one frame with its
// scratch in a fixed array that is part of this library's device image:
// every GPU that loads the library holds LACOS_STATIC_SCRATCH_BYTES for it
// until the process exits, and no call allocates or frees anything.
namespace {

__device__ __align__(256) unsigned char g_static_scratch[LACOS_STATIC_SCRATCH_BYTES];

struct StaticDevice {
  bool ready = false;
  void* scratch = nullptr;  // device address of g_static_scratch on this device
  int num_sms = 0, bpsm_core[2] = {1, 1}, bpsm_final[2] = {1, 1}, core_variant = kDefaultCoreVariant;
};
std::mutex g_static_mu;
constexpr int kStaticMaxDevices = 64;
StaticDevice g_static_dev[kStaticMaxDevices];

__global__ void store_desc_kernel(FrameDesc* dst, FrameDesc d) { *dst = d; }

// Once per device, with that device current: the array's device address
// (a host-side name of a __device__ array is not a device pointer) and the
// launch geometry.
cudaError_t static_setup(int dev, StaticDevice*& out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticDevice& sd = g_static_dev[dev];
  if (!sd.ready) {
    cudaError_t e = cudaGetSymbolAddress(&sd.scratch, g_static_scratch);
    if (e != cudaSuccess) return e;
    if (const char* env = std::getenv("LACOS_CORE_VARIANT")) {
      const int v = std::atoi(env);
      if (v >= 0 && v < LACOS_CORE_VARIANTS) sd.core_variant = v;
    }
    const CoreVariant& V = kCoreVariants[sd.core_variant];
    e = cudaDeviceGetAttribute(&sd.num_sms, cudaDevAttrMultiProcessorCount, dev);
    for (int dt = 0; dt < 2 && e == cudaSuccess; ++dt) {
      e = cudaFuncSetAttribute(V.fn[dt], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)V.smem[dt]);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sd.bpsm_core[dt], V.fn[dt], V.nt, V.smem[dt]);
      sd.bpsm_core[dt] = std::max(1, sd.bpsm_core[dt]);
    }
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sd.bpsm_final[0], finalize_kernel<FGSmall>, kBlock, 0);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sd.bpsm_final[1], finalize_kernel<FGBig>, kBlock, 0);
    if (e != cudaSuccess) return e;
    for (int& b : sd.bpsm_final) b = std::max(1, b);
    sd.ready = true;
  }
  out = &sd;
  return cudaSuccess;
}

}  // namespace

extern "C" int lacos_run_static(const void* d_frame, lacos_dtype dt, int ny, int nx,
                                const lacos_params* p, uint8_t* d_mask, float* d_clean,
                                lacos_stream stream, lacos_result* res) {
  const auto t_call = std::chrono::steady_clock::now();
  if (!p) return LACOS_EINVAL;
  const FrameReq f{d_frame, (int)dt, ny, nx, *p, d_mask, d_clean};
  if (!frame_valid(f)) return LACOS_EINVAL;
  // The same layout as a one-frame request (heads, descriptor, state, five
  // bit-planes), computed without touching the heap.
  const size_t mb = maskbuf_bytes(ny, nx);
  const size_t off_desc = align_up(sizeof(unsigned) * kHeads);
  const size_t off_state = off_desc + align_up(sizeof(FrameDesc));
  const size_t off_masks = off_state + align_up(sizeof(FrameState));
  const size_t need = off_masks + (p->satgrow ? 6 : 5) * mb + kNtabBytes + tflag_bytes(ny, nx) +
                      (p->gain == 0.0f ? kGainHistBytes : 0);
  if (need > (size_t)LACOS_STATIC_SCRATCH_BYTES) return LACOS_ENOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return LACOS_ECUDA;
  StaticDevice* sd = nullptr;
  if (static_setup(dev, sd) != cudaSuccess) return LACOS_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  char* d = (char*)sd->scratch;
  unsigned* heads = (unsigned*)d;
  FrameDesc* ddesc = (FrameDesc*)(d + off_desc);
  FrameState* dstate = (FrameState*)(d + off_state);
  char* planes = d + off_masks;

  FrameDesc h;
  std::memset(&h, 0, sizeof(h));
  h.x0 = f.frame;
  h.dtype = f.dtype;
  h.ny = ny;
  h.nx = nx;
  h.wpr = wpr_of(nx);
  h.mbuf0 = (uint32_t*)planes;
  h.mbuf1 = (uint32_t*)(planes + mb);
  h.p_sig = (uint32_t*)(planes + 2 * mb);
  h.p_lo = (uint32_t*)(planes + 3 * mb);
  h.p_cand = (uint32_t*)(planes + 4 * mb);
  h.ntab = (float2*)(planes + 5 * mb);
  h.tflags = (uint8_t*)(planes + 5 * mb + kNtabBytes);
  char* after = planes + 5 * mb + kNtabBytes + tflag_bytes(ny, nx);
  h.p_sat = p->satgrow ? (uint32_t*)after : nullptr;
  if (p->satgrow) after += mb;
  h.ghist_n = p->gain == 0.0f ? (unsigned*)after : nullptr;
  h.ghist_a = p->gain == 0.0f ? (unsigned long long*)(after + kGainHistN) : nullptr;
  h.mask_out = d_mask;
  h.clean_out = d_clean;
  h.st = dstate;
  h.gain = p->gain;
  h.gain_est = p->gain == 0.0f;
  h.rn = p->readnoise;
  volatile float rn = p->readnoise;
  volatile float rn2 = rn * rn;
  h.rn2 = rn2;
  h.satlevel = p->satlevel;
  h.sigclip = p->sigclip;
  volatile float lo = p->sigfrac * p->sigclip;
  h.lo = lo;
  h.thr_min = std::min(h.lo, h.sigclip);
  h.objlim = p->objlim;
  h.niter = p->niter;
  h.fnorm = p->fine_norm;
  h.satgrow = p->satgrow;
  h.sepmed = p->sepmed;
  const CoreVariant& V = kCoreVariants[sd->core_variant];
  h.th = V.th;
  h.tw = V.tw;
  h.tiles_x = (nx + V.tw - 1) / V.tw;
  const unsigned total = (unsigned)h.tiles_x * (unsigned)((ny + V.th - 1) / V.th);
  h.tile_begin = 0;
  h.tile_end = total;
  const PassShapes ps = pass_shapes((unsigned long long)ny * (unsigned long long)nx);
  h.ftiles_x = (nx + ps.ftw - 1) / ps.ftw;
  const unsigned total_fin = (unsigned)h.ftiles_x * (unsigned)((ny + ps.fth - 1) / ps.fth);
  h.fin_begin = 0;
  h.fin_end = total_fin;
  h.word_begin = 0;
  h.gblk_x = (unsigned)((h.wpr + ps.gw - 1) / ps.gw);
  h.gblk_begin = 0;
  const unsigned total_gblk = h.gblk_x * (unsigned)((ny + ps.gh - 1) / ps.gh);

  // The array keeps the previous call's contents: the descriptor is
  // rewritten, and the queue heads, the state and M_0 are cleared.
  store_desc_kernel<<<1, 1, 0, s>>>(ddesc, h);
  if (cudaGetLastError() != cudaSuccess) return LACOS_ECUDA;
  if (cudaMemsetAsync(heads, 0, sizeof(unsigned) * kHeads, s) != cudaSuccess ||
      cudaMemsetAsync(dstate, 0, sizeof(FrameState), s) != cudaSuccess ||
      cudaMemsetAsync(h.mbuf0, 0, mb, s) != cudaSuccess ||
      cudaMemsetAsync(h.tflags, 0, tflag_bytes(ny, nx), s) != cudaSuccess ||
      (h.ghist_n && cudaMemsetAsync(h.ghist_n, 0, kGainHistBytes, s) != cudaSuccess))
    return LACOS_ECUDA;
  const int di = f.dtype == LACOS_U16 ? 1 : 0;
  const unsigned gd = std::min<unsigned>(total, (unsigned)(sd->num_sms * sd->bpsm_core[di]));
  const unsigned gfi = std::min<unsigned>(total_fin, (unsigned)(sd->num_sms * sd->bpsm_final[ps.big]));
  ntab_kernel<<<dim3(256, 1), 256, 0, s>>>(ddesc, 1);
  if (p->satgrow) {
    const unsigned nw = (unsigned)((size_t)ny * wpr_of(nx));
    satseed_kernel<<<(nw + 255) / 256, 256, 0, s>>>(ddesc, 0, nw);
    satgrow_kernel<<<(nw + 255) / 256, 256, 0, s>>>(ddesc, 0, nw);
  }
  for (int k = 1; k <= p->niter; ++k) {
    if (h.gain_est) launch_gain_level(ddesc, 1, k, sd->num_sms, s);
    V.fn[di]<<<gd, V.nt, V.smem[di], s>>>(ddesc, 1, 0, total, k, heads + kHeadCore + di * kHeadLevels + k);
    launch_grow(ps.big, total_gblk, ddesc, 1, k, s);
  }
  launch_finalize(ps.big, gfi, ddesc, 1, total_fin, heads + kHeadFinal, s);
  if (cudaGetLastError() != cudaSuccess) return LACOS_ECUDA;
  FrameState hs;
  if (cudaMemcpyAsync(&hs, dstate, sizeof(FrameState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LACOS_ECUDA;
  if (res) {
    res->status = (hs.err & ERR_NONFINITE)  ? LACOS_ENONFINITE
                  : (hs.err & ERR_TIMEOUT) ? LACOS_ETIMEOUT
                  : (hs.err & ERR_NOGAIN)  ? LACOS_ENOGAIN
                                           : LACOS_OK;
    res->gain = h.gain_est ? hs.gain : p->gain;
    res->iters_run = hs.iters_run;
    res->n_flagged = (long long)hs.flagged;
    // The call blocks until its work is done: its latency is the host time
    // from entry to completion (queueing behind earlier work on `stream`
    // included).
    res->latency_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_call).count();
  }
  return LACOS_OK;
}
