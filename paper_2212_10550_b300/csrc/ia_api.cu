// C ABI of the articulated radiance-field render path (see include/ia.h).
//
// Host side only: argument checks, device memory owned by the context, and
// kernel launches.  Every entry point returns an ia_status and records a
// message on failure; nothing here aborts the process.
#include <cmath>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ia.h"
#include "../../include/ia_measure.h"
#include "ia_internal.h"

using namespace ia;

constexpr int kBoxListCap = 64;  // boxes remembered per occupied cell (about 52 on average at full size)

struct ia_ctx {
  ia_config cfg{};
  int device = 0;
  int num_sms = 0;
  std::string err;
  // skeleton
  int nb = 0;
  int Rw = 0;
  float cmin[3]{}, cmax[3]{}, nmin[3]{}, nmax[3]{};
  int* d_parent = nullptr;
  double* d_rest = nullptr;
  float* d_skin = nullptr;
  // canonical field
  int n_in = 0;
  int64_t n_entries = 0;
  Level levels[kMaxLevels]{};
  float* d_table = nullptr;
  __half2* d_table_h = nullptr;  // fp16 shadow (reduced-precision field only)
  float* d_mlp = nullptr;
  bool have_params = false;
  // poses
  int n_poses = 0, pose_cap = 0;
  float* d_N = nullptr;
  float* d_Ninv = nullptr;
  float* d_B0inv = nullptr;
  float4* d_M = nullptr;
  double* d_theta = nullptr;
  double* d_trans = nullptr;
  // occupancy
  uint32_t* d_occ = nullptr;
  uint32_t* d_occ_train = nullptr;
  float* d_sigma = nullptr;
  float* d_occ_ema = nullptr;  // training-mode running density [R^3] (zero at creation)
  // root culling: per occupancy cell a 64-bit mask of the sub-cells where a root
  // is possible, for pose sub_pose (-1: none; any change of the blended grid
  // clears it), and the occupancy cells to search
  unsigned long long* d_sub = nullptr;  // [R^3]
  unsigned* d_cen = nullptr;             // [ceil(R^3 / 32)] centre flags of the culling
  unsigned* d_cand_count = nullptr;
  int* d_cand = nullptr;                // [R^3]
  int sub_pose = -1;
  bool occ_cull = true;
  // the grown image box of every skinning cell for pose box_pose (written with
  // the culling masks of a per-pose refresh), and per occupied cell of d_occ
  // the boxes meeting it, valid for pose blist_pose (rebuilt whenever d_occ is
  // written with valid boxes; -1 otherwise)
  float4* d_cell_box = nullptr;          // [(Rw - 1)^3][2]
  int* d_blist_count = nullptr;          // [R^3]
  int* d_blist = nullptr;                // [R^3][kBoxListCap]
  int box_pose = -1, blist_pose = -1;
  // the same masks for every pose, for the training step: [sub_all_cap][R^3]
  unsigned long long* d_sub_all = nullptr;
  int sub_all_cap = 0;
  bool sub_all_valid = false;
  // with the proposal search: every pose's grown boxes and, per cell of the
  // grid, the boxes meeting it (the training step's fallback point test),
  // valid with the masks
  float4* d_tcell_box = nullptr;   // [tblist_cap][(Rw - 1)^3][2]
  int* d_tblist_count = nullptr;   // [tblist_cap][R^3]
  int* d_tblist = nullptr;         // [tblist_cap][R^3][kBoxListCap]
  int tblist_cap = 0;
  bool tblist_valid = false;
  bool have_occ = false;
  // counters
  unsigned long long* d_stats = nullptr;
  unsigned int* d_counter = nullptr;
  unsigned int* d_work = nullptr;   // list counters: [0] occupancy, [1] training sample kernel
  unsigned long long* d_tstats = nullptr;  // counters of the last training step
  // scratch for host-memory outputs of ia_render
  float* d_out = nullptr;
  size_t out_cap = 0;
  // wavefront render path: per-ray and per-sample arrays, counters
  int render_path = IA_RENDER_WAVEFRONT;
  size_t wf_ray_cap = 0, wf_cap = 0;
  size_t wf_i0_cap = 0;  // float4s in d_wf_item0
  size_t wf_pcap = 0;    // samples in the proposal arrays (d_wf_prop, d_wf_fb, d_wf_fbidx; d_wf_item1 x n_bones)
  int* d_wf_first = nullptr;
  int* d_wf_cnt = nullptr;
  float* d_wf_dt = nullptr;
  float4* d_wf_xn = nullptr;
  float4* d_wf_prop = nullptr;
  float4* d_wf_item0 = nullptr;
  float4* d_wf_item1 = nullptr;
  int* d_wf_fb = nullptr;
  int* d_wf_fbidx = nullptr;
  float4* d_wf_res = nullptr;
  unsigned* d_wf_counts = nullptr;  // [0] samples, [1] fallback samples
  // the occupancy density's query points and results (R^3 each)
  size_t wf_occ_cap = 0;
  float4* d_wf_oxn = nullptr;
  float4* d_wf_ores = nullptr;
  // training-step workspace
  int ray_cap = 0;
  int reg_cap = 0;
  ia_loss loss{IA_LOSS_L2, 0.f, 1.f, 0.f, 0.f};
  // Adam state of the canonical field (table then MLP, one allocation each)
  float* d_fm = nullptr;
  float* d_fv = nullptr;
  int field_step = 0;
  float* d_sm = nullptr;  // Adam state of the skinning-weight grid
  float* d_sv = nullptr;
  int skin_step = 0;
  int* d_reg_idx = nullptr;
  int* d_ray_n = nullptr;
  float* d_ray_dt = nullptr;
  int* d_ray_idx = nullptr;
  int* d_count = nullptr;
  size_t s_cap = 0;
  float4* d_s_pos = nullptr;
  float4* d_s_out = nullptr;
  float4* d_s_x = nullptr;
  float4* d_s_grad = nullptr;
  float4* d_s_dfeat = nullptr;
  float4* d_s_gx = nullptr;
  float* d_act = nullptr;           // fp32 step: per-sample activations
  uint16_t* d_X = nullptr;          // fp16 / bf16 step: channel-major GEMM operands
  int64_t x_ld = 0;
  CUtensorMap x_map{};
  float* d_scale = nullptr;         // loss scale, the step's skip flags, clean steps
  int* d_overflow = nullptr;
  int* d_good = nullptr;
  uint64_t wait_ns = kDefaultWaitNs;  // bound on each wait of the tensor-core pipeline
  // the last ia_train_forward, kept for its ia_train_backward
  bool fwd_valid = false;
  bool fwd_own_params = false;  // it read the context's own table / MLP
  TrainArgs fwd{};
  __half2* d_table_h_ext = nullptr;  // fp16 shadow of a caller table (reduced-precision forward)
  int inject = 0;                     // ia_set_fault_injection flags
  // proposal network
  bool prop_ready = false;
  int search = IA_SEARCH_ALL_BONES;
  ia_proposal_config pcfg{};
  Level plv[kMaxLevels]{};
  int64_t p_entries = 0, p_mlp = 0;
  float* d_pp = nullptr;      // parameters: table then MLP (one allocation)
  float* d_ptable = nullptr;  // views into d_pp
  float* d_pmlp = nullptr;
  float* d_ploss = nullptr;   // scratch loss of training steps
  float* d_pg = nullptr;   // gradients: table then MLP
  float* d_pm = nullptr;   // Adam first moments (same layout)
  float* d_pv = nullptr;   // Adam second moments
  int adam_step = 0;
  int prow_cap = 0;
  float* d_prows = nullptr;
  int pair_cap = 0;
  int pose_ws_cap = 0;
  int* d_pose_ws = nullptr;   // training step: per-pose sample totals / offsets and fill counters
  int pb1_cap = 0;
  float* d_pb1 = nullptr;     // per-pose layer-1 bias of the training step's proposal
  float* d_pxc = nullptr;
  int* d_pstart = nullptr;
};

namespace {

thread_local std::string g_create_err;

ia_status fail(ia_ctx* c, ia_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_err = buf;
  return st;
}

ia_status cuda_fail(ia_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so the next call starts clean
  if (e == cudaErrorMemoryAllocation) return fail(c, IA_ERR_OOM, "%s: out of device memory", what);
  return fail(c, IA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define IA_CUDA(c, call, what)                      \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail((c), e_, (what)); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

bool finite3(const float v[3]) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

FieldDev field_dev(const ia_ctx* c) {
  FieldDev F{};
  F.table = reinterpret_cast<const float2*>(c->d_table);
  F.L = c->cfg.n_levels;
  for (int l = 0; l < kMaxLevels; ++l) F.lv[l] = c->levels[l];
  for (int a = 0; a < 3; ++a) {
    F.cmin[a] = c->cmin[a];
    F.inv_ext[a] = 1.0f / (c->cmax[a] - c->cmin[a]);
  }
  return F;
}

PropDev prop_dev(const ia_ctx* c) {
  PropDev Q{};
  if (!c->prop_ready) return Q;
  Q.table = reinterpret_cast<const float2*>(c->d_ptable);
  Q.L = c->pcfg.n_levels;
  for (int l = 0; l < kMaxLevels; ++l) Q.lv[l] = c->plv[l];
  for (int a = 0; a < 3; ++a) {
    Q.nmin[a] = c->nmin[a];
    Q.inv_ext[a] = 1.0f / (c->nmax[a] - c->nmin[a]);
  }
  Q.mlp = c->d_pmlp;
  Q.n_in = 2 * c->pcfg.n_levels + 3 * c->nb;
  Q.top_k = c->pcfg.top_k;
  return Q;
}

PosedArgs posed_args(const ia_ctx* c, int pose) {
  PosedArgs a{};
  a.S.M = c->d_M + (size_t)pose * c->Rw * c->Rw * c->Rw * 3;
  a.S.Rw = c->Rw;
  for (int i = 0; i < 3; ++i) {
    a.S.cmin[i] = c->cmin[i];
    a.S.cmax[i] = c->cmax[i];
    a.S.scale[i] = (float)(c->Rw - 1) / (c->cmax[i] - c->cmin[i]);
  }
  a.F = field_dev(c);
  a.cfg.nb = c->nb;
  a.cfg.max_iter = c->cfg.broyden_max_iter;
  a.cfg.tol2 = c->cfg.broyden_tol * c->cfg.broyden_tol;
  a.Ninv = c->d_Ninv + (size_t)pose * c->nb * 12;
  a.mlp = c->d_mlp;
  a.n_in = c->n_in;
  a.prec = c->cfg.precision;
  a.table_h = c->d_table_h;
  a.search = (c->search == IA_SEARCH_PROPOSAL && c->prop_ready && c->cfg.precision != IA_FP32) ? 1 : 0;
  a.prop = prop_dev(c);
  a.theta = c->d_theta ? c->d_theta + (size_t)pose * c->nb * 3 : nullptr;
  return a;
}

// Occupancy cells take the context's search.  (Without culling most searched
// cells were empty space, where the proposal's starts find nothing and every
// bone-wise start runs anyway; with culling most searched cells have a root.)
PosedArgs occ_args(const ia_ctx* c, int pose) { return posed_args(c, pose); }

// field-only arguments (no pose needed)
PosedArgs posed_args_params(const ia_ctx* c) {
  PosedArgs a{};
  a.F = field_dev(c);
  a.mlp = c->d_mlp;
  a.n_in = c->n_in;
  a.prec = c->cfg.precision;
  a.table_h = c->d_table_h;
  return a;
}

BoxDev box_dev(const ia_ctx* c) {
  BoxDev b{};
  b.R = c->cfg.occ_res;
  for (int a = 0; a < 3; ++a) {
    b.nmin[a] = c->nmin[a];
    b.nmax[a] = c->nmax[a];
    const float ext = c->nmax[a] - c->nmin[a];  // fp32, as the documented indexing
    b.cell_scale[a] = (float)b.R / ext;
    b.cell_size[a] = ext / (float)b.R;
    b.sub_scale[a] = (float)(kSub * b.R) / ext;
  }
  return b;
}

// Density of the posed field at every occupancy cell's query point (centre, or
// norm_min + (c + jitter) * cell size) into sigma [R^3]: with culling on, only
// the cells whose point can have a root are searched, the rest get 0 (the same
// values the full search gives).
// The culling masks built here stay valid for the render of the same pose.
// Item arrays of the search waves for chunks of up to cap samples (kept
// across calls; grown, never shrunk).
ia_status ensure_wf_items(ia_ctx* c, size_t cap, int per0, bool prop, cudaStream_t s) {
  if (cap == 0) return IA_OK;
  if (cap * per0 > c->wf_i0_cap || (prop && cap > c->wf_pcap)) IA_CUDA(c, cudaStreamSynchronize(s), "wavefront arrays");
  if (cap * per0 > c->wf_i0_cap) {
    c->wf_i0_cap = 0;
    IA_CUDA(c, dalloc(&c->d_wf_item0, cap * per0), "wavefront arrays");
    c->wf_i0_cap = cap * per0;
  }
  if (prop && cap > c->wf_pcap) {
    c->wf_pcap = 0;
    IA_CUDA(c, dalloc(&c->d_wf_prop, cap), "wavefront arrays");
    IA_CUDA(c, dalloc(&c->d_wf_item1, cap * c->nb), "wavefront arrays");
    IA_CUDA(c, dalloc(&c->d_wf_fb, cap), "wavefront arrays");
    IA_CUDA(c, dalloc(&c->d_wf_fbidx, cap), "wavefront arrays");
    c->wf_pcap = cap;
  }
  if (!c->d_wf_counts) IA_CUDA(c, dalloc(&c->d_wf_counts, (size_t)2), "wavefront arrays");
  return IA_OK;
}

// The search and field run on the wavefront kernels over arrays the context
// keeps for R^3 samples; with fixed_memory (the allocation-free entry) on the
// fused density kernel, whose lanes run each cell's starts in the same order
// with the same arithmetic: the same densities bit for bit.
cudaError_t occ_density(ia_ctx* c, int pose, const float* jitter, float* sigma, unsigned long long* stats,
                        cudaStream_t s, bool fixed_memory) {
  const PosedArgs a = occ_args(c, pose);
  const BoxDev box = box_dev(c);
  WfArgs w{};
  if (!fixed_memory) {
    const size_t n_all = (size_t)box.R * box.R * box.R;
    const bool prop = a.search != 0;
    const int per0 = prop ? std::min(c->pcfg.top_k, c->nb) : c->nb;
    if (c->wf_occ_cap < n_all) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return e;
      c->wf_occ_cap = 0;
      if ((e = dalloc(&c->d_wf_oxn, n_all)) != cudaSuccess) return e;
      if ((e = dalloc(&c->d_wf_ores, n_all)) != cudaSuccess) return e;
      c->wf_occ_cap = n_all;
    }
    if (ensure_wf_items(c, n_all, per0, prop, s) != IA_OK) return cudaErrorMemoryAllocation;
    w.xn = c->d_wf_oxn;
    w.res = c->d_wf_ores;
    w.cap = (int)n_all;
    w.prop = c->d_wf_prop;
    w.item0 = c->d_wf_item0;
    w.item1 = c->d_wf_item1;
    w.fb = c->d_wf_fb;
    w.fbidx = c->d_wf_fbidx;
    w.n_fb = c->d_wf_counts + 1;
  }
  auto density = [&](const int* cells, const unsigned* count) {
    return fixed_memory ? launch_occ_density(a, box, jitter, cells, count, sigma, stats, c->d_work, c->num_sms, s)
                        : launch_wf_occupancy(a, box, jitter, cells, count, sigma, stats, w, c->num_sms, s);
  };
  if (!c->occ_cull) return density(nullptr, nullptr);
  c->sub_pose = -1;
  c->box_pose = -1;
  c->blist_pose = -1;
  // the boxes themselves only serve the proposal search's fallback test
  float4* cell_box = a.search ? c->d_cell_box : nullptr;
  cudaError_t e = launch_occ_cull(a, box, jitter, c->d_sub, c->d_cen, c->d_cand_count, c->d_cand, sigma, stats, s,
                                  cell_box);
  if (e != cudaSuccess) return e;
  c->sub_pose = pose;
  c->box_pose = cell_box ? pose : -1;
  return density(c->d_cand, c->d_cand_count);
}

// The box lists of the grid just written to d_occ, when the boxes belong to a
// pose (a per-pose refresh with culling computed them); otherwise none.
static cudaError_t rebuild_box_lists(ia_ctx* c, cudaStream_t s) {
  c->blist_pose = -1;
  if (!c->occ_cull || c->box_pose < 0 || !c->d_cell_box) return cudaSuccess;
  const int nc = c->Rw - 1;
  cudaError_t e = launch_occ_boxlist(c->d_cell_box, nc * nc * nc, 1, box_dev(c), c->d_occ, c->d_blist_count,
                                     c->d_blist, kBoxListCap, s);
  if (e == cudaSuccess) c->blist_pose = c->box_pose;
  return e;
}

ia_status need_ready(ia_ctx* c, int pose, bool need_occ) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (c->nb == 0) return fail(c, IA_ERR_STATE, "ia_set_skeleton has not been called");
  if (!c->have_params) return fail(c, IA_ERR_STATE, "ia_set_params has not been called");
  if (c->n_poses == 0) return fail(c, IA_ERR_STATE, "ia_set_pose has not been called");
  if (pose < 0 || pose >= c->n_poses) return fail(c, IA_ERR_ARG, "pose %d out of range [0, %d)", pose, c->n_poses);
  if (need_occ && !c->have_occ) return fail(c, IA_ERR_STATE, "no occupancy grid (ia_update_occupancy first)");
  return IA_OK;
}

void read_stats(ia_ctx* c, ia_render_stats* out, cudaStream_t s, const unsigned long long* src = nullptr) {
  unsigned long long h[ST_COUNT];
  cudaMemcpyAsync(h, src ? src : c->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  out->rays = (int64_t)h[ST_RAYS];
  out->hit_rays = (int64_t)h[ST_HIT];
  out->marched_slots = (int64_t)h[ST_MARCHED];
  out->occupied_samples = (int64_t)h[ST_OCC];
  out->starts = (int64_t)h[ST_STARTS];
  out->broyden_iters = (int64_t)h[ST_ITERS];
  out->converged = (int64_t)h[ST_CONV];
  out->roots = (int64_t)h[ST_ROOTS];
  out->early_stopped = (int64_t)h[ST_EARLY];
  out->proposed = (int64_t)h[ST_PROP];
  out->fallbacks = (int64_t)h[ST_FALLBACK];
  out->culled = (int64_t)h[ST_CULLED];
  out->grid_gathers = (int64_t)h[ST_GATHERS];
  out->rooted_samples = (int64_t)h[ST_ROOTED];
  out->point_culled = (int64_t)h[ST_PCULLED];
}

}  // namespace

extern "C" {

const char* ia_version(void) { return "ia-b300 0.1 (sm_103a)"; }

const char* ia_last_error(const ia_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

ia_status ia_create(const ia_config* cfg, ia_ctx** out) {
  if (!cfg || !out) return fail(nullptr, IA_ERR_ARG, "null argument");
  *out = nullptr;
  const ia_config& g = *cfg;
  if (g.n_levels < 1 || g.n_levels > IA_MAX_LEVELS) return fail(nullptr, IA_ERR_ARG, "n_levels must be 1..16");
  if (g.n_features != 2) return fail(nullptr, IA_ERR_ARG, "n_features must be 2");
  if (g.log2_table < 10 || g.log2_table > 24) return fail(nullptr, IA_ERR_ARG, "log2_table must be 10..24");
  for (int l = 0; l < g.n_levels; ++l)
    if (g.level_res[l] < 2 || g.level_res[l] > (1 << 20))
      return fail(nullptr, IA_ERR_ARG, "level_res[%d] = %d outside 2..2^20", l, g.level_res[l]);
  if (g.mlp_width != 64) return fail(nullptr, IA_ERR_ARG, "mlp_width must be 64");
  if (g.max_samples < 1 || g.max_samples > 1024) return fail(nullptr, IA_ERR_ARG, "max_samples must be 1..1024");
  if (g.broyden_max_iter < 1 || g.broyden_max_iter > 64)
    return fail(nullptr, IA_ERR_ARG, "broyden_max_iter must be 1..64");
  if (!(g.broyden_tol > 0.f) || !std::isfinite(g.broyden_tol)) return fail(nullptr, IA_ERR_ARG, "broyden_tol must be > 0");
  if (g.occ_res < 2 || g.occ_res > 256) return fail(nullptr, IA_ERR_ARG, "occ_res must be 2..256");
  if (!std::isfinite(g.occ_tau)) return fail(nullptr, IA_ERR_ARG, "occ_tau must be finite");
  if (g.occ_dilate < 0 || g.occ_dilate > 4) return fail(nullptr, IA_ERR_ARG, "occ_dilate must be 0..4");
  if (!std::isfinite(g.early_stop_T) || g.early_stop_T >= 1.f)
    return fail(nullptr, IA_ERR_ARG, "early_stop_T must be finite and < 1");
  if (g.precision != IA_FP32 && g.precision != IA_FP16 && g.precision != IA_BF16)
    return fail(nullptr, IA_ERR_ARG, "precision %d not available", g.precision);

  ia_ctx* c = new ia_ctx();
  c->cfg = g;
  cudaGetDevice(&c->device);
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(nullptr, IA_ERR_CUDA, "no usable CUDA device");
  }
  const int64_t T = 1LL << g.log2_table;
  int64_t off = 0;
  for (int l = 0; l < g.n_levels; ++l) {
    const int64_t r1 = (int64_t)g.level_res[l] + 1;
    const int64_t dense = r1 * r1 * r1;
    Level& lv = c->levels[l];
    lv.res = g.level_res[l];
    lv.dense = dense <= T ? 1 : 0;
    lv.size = (uint32_t)(dense <= T ? dense : T);
    lv.offset = (uint32_t)off;
    off += lv.size;
  }
  c->n_entries = off;
  c->n_in = 2 * g.n_levels;
  const int R = g.occ_res;
  const size_t words = ((size_t)R * R * R + 31) / 32;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dalloc(&c->d_table, (size_t)off * 2);
  if (e == cudaSuccess && g.precision != IA_FP32) e = dalloc(&c->d_table_h, (size_t)off);
  if (e == cudaSuccess) e = dalloc(&c->d_mlp, (size_t)kWidth * c->n_in + kWidth + kWidth * kWidth + kWidth + 4 * kWidth + 4);
  if (e == cudaSuccess) e = dalloc(&c->d_occ, words);
  if (e == cudaSuccess) e = dalloc(&c->d_occ_train, words);
  if (e == cudaSuccess) e = dalloc(&c->d_sigma, (size_t)R * R * R);
  if (e == cudaSuccess) e = dalloc(&c->d_occ_ema, (size_t)R * R * R);
  if (e == cudaSuccess) e = dalloc(&c->d_sub, (size_t)R * R * R);
  if (e == cudaSuccess) e = dalloc(&c->d_cen, ((size_t)R * R * R + 31) / 32);
  if (e == cudaSuccess) e = dalloc(&c->d_cand_count, (size_t)1);
  if (e == cudaSuccess) e = dalloc(&c->d_blist_count, (size_t)R * R * R);
  if (e == cudaSuccess) e = dalloc(&c->d_blist, (size_t)R * R * R * kBoxListCap);
  if (e == cudaSuccess) e = dalloc(&c->d_cand, (size_t)R * R * R);
  if (e == cudaSuccess) e = cudaMemset(c->d_occ_ema, 0, sizeof(float) * R * R * R);
  if (e == cudaSuccess) e = dalloc(&c->d_stats, (size_t)ST_COUNT);
  if (e == cudaSuccess) e = dalloc(&c->d_counter, (size_t)1);
  if (e == cudaSuccess) e = dalloc(&c->d_work, (size_t)2);
  if (e == cudaSuccess) e = dalloc(&c->d_tstats, (size_t)ST_COUNT);
  if (e == cudaSuccess) e = cudaMemset(c->d_tstats, 0, sizeof(unsigned long long) * ST_COUNT);
  if (e == cudaSuccess) e = cudaMemset(c->d_occ_train, 0, words * sizeof(uint32_t));
  if (e != cudaSuccess) {
    ia_status st = cuda_fail(nullptr, e, "ia_create");
    ia_destroy(c);
    return st;
  }
  *out = c;
  return IA_OK;
}

void ia_destroy(ia_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  dfree(c->d_parent);
  dfree(c->d_rest);
  dfree(c->d_skin);
  dfree(c->d_table);
  dfree(c->d_table_h);
  dfree(c->d_mlp);
  dfree(c->d_N);
  dfree(c->d_Ninv);
  dfree(c->d_B0inv);
  dfree(c->d_M);
  dfree(c->d_theta);
  dfree(c->d_trans);
  dfree(c->d_occ);
  dfree(c->d_occ_train);
  dfree(c->d_sigma);
  dfree(c->d_occ_ema);
  dfree(c->d_sub);
  dfree(c->d_cen);
  dfree(c->d_sub_all);
  dfree(c->d_tcell_box);
  dfree(c->d_tblist_count);
  dfree(c->d_tblist);
  dfree(c->d_cand_count);
  dfree(c->d_blist_count);
  dfree(c->d_blist);
  dfree(c->d_cell_box);
  dfree(c->d_cand);
  dfree(c->d_stats);
  dfree(c->d_counter);
  dfree(c->d_wf_first);
  dfree(c->d_wf_cnt);
  dfree(c->d_wf_dt);
  dfree(c->d_wf_xn);
  dfree(c->d_wf_prop);
  dfree(c->d_wf_item0);
  dfree(c->d_wf_item1);
  dfree(c->d_wf_fb);
  dfree(c->d_wf_fbidx);
  dfree(c->d_wf_res);
  dfree(c->d_wf_counts);
  dfree(c->d_wf_oxn);
  dfree(c->d_wf_ores);
  dfree(c->d_work);
  dfree(c->d_tstats);
  dfree(c->d_out);
  dfree(c->d_ray_n);
  dfree(c->d_ray_dt);
  dfree(c->d_ray_idx);
  dfree(c->d_reg_idx);
  dfree(c->d_fm);
  dfree(c->d_fv);
  dfree(c->d_sm);
  dfree(c->d_sv);
  dfree(c->d_count);
  dfree(c->d_s_pos);
  dfree(c->d_s_out);
  dfree(c->d_s_x);
  dfree(c->d_s_grad);
  dfree(c->d_s_dfeat);
  dfree(c->d_s_gx);
  dfree(c->d_act);
  dfree(c->d_X);
  dfree(c->d_scale);
  dfree(c->d_overflow);
  dfree(c->d_table_h_ext);
  dfree(c->d_good);
  dfree(c->d_pp);
  dfree(c->d_ploss);
  dfree(c->d_pg);
  dfree(c->d_pm);
  dfree(c->d_pv);
  dfree(c->d_prows);
  dfree(c->d_pxc);
  dfree(c->d_pb1);
  dfree(c->d_pose_ws);
  dfree(c->d_pstart);
  delete c;
}

ia_status ia_set_skeleton(ia_ctx* c, int n_bones, const int32_t* parent, const double* rest_joints,
                          const float* skin_grid, int skin_res, const float canon_min[3], const float canon_max[3],
                          const float norm_min[3], const float norm_max[3]) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (n_bones < 1 || n_bones > IA_MAX_BONES) return fail(c, IA_ERR_ARG, "n_bones must be 1..%d", IA_MAX_BONES);
  if (!parent || !rest_joints || !skin_grid || !canon_min || !canon_max || !norm_min || !norm_max)
    return fail(c, IA_ERR_ARG, "null argument");
  if (skin_res < 2 || skin_res > 256) return fail(c, IA_ERR_ARG, "skin_res must be 2..256");
  if (parent[0] != -1) return fail(c, IA_ERR_ARG, "parent[0] must be -1 (bone 0 is the root)");
  for (int k = 1; k < n_bones; ++k)
    if (parent[k] < 0 || parent[k] >= k)
      return fail(c, IA_ERR_ARG, "parent[%d] = %d: parents must precede children", k, parent[k]);
  for (int i = 0; i < 3 * n_bones; ++i)
    if (!std::isfinite(rest_joints[i])) return fail(c, IA_ERR_ARG, "rest_joints must be finite");
  if (!finite3(canon_min) || !finite3(canon_max) || !finite3(norm_min) || !finite3(norm_max))
    return fail(c, IA_ERR_ARG, "boxes must be finite");
  for (int a = 0; a < 3; ++a)
    if (!(canon_max[a] > canon_min[a]) || !(norm_max[a] > norm_min[a]))
      return fail(c, IA_ERR_ARG, "box max must exceed min on every axis");
  const size_t V = (size_t)skin_res * skin_res * skin_res;
  IA_CUDA(c, dalloc(&c->d_parent, (size_t)n_bones), "ia_set_skeleton");
  IA_CUDA(c, dalloc(&c->d_rest, (size_t)3 * n_bones), "ia_set_skeleton");
  IA_CUDA(c, dalloc(&c->d_skin, V * n_bones), "ia_set_skeleton");
  IA_CUDA(c, dalloc(&c->d_cell_box, (size_t)2 * (skin_res - 1) * (skin_res - 1) * (skin_res - 1)), "ia_set_skeleton");
  IA_CUDA(c, cudaMemcpy(c->d_parent, parent, sizeof(int) * n_bones, cudaMemcpyHostToDevice), "ia_set_skeleton");
  IA_CUDA(c, cudaMemcpy(c->d_rest, rest_joints, sizeof(double) * 3 * n_bones, cudaMemcpyHostToDevice),
          "ia_set_skeleton");
  IA_CUDA(c, cudaMemcpy(c->d_skin, skin_grid, sizeof(float) * V * n_bones, cudaMemcpyDefault), "ia_set_skeleton");
  if (c->d_sm) {  // a new grid: its Adam state restarts
    dfree(c->d_sm);
    dfree(c->d_sv);
    c->skin_step = 0;
  }
  c->nb = n_bones;
  c->Rw = skin_res;
  for (int a = 0; a < 3; ++a) {
    c->cmin[a] = canon_min[a];
    c->cmax[a] = canon_max[a];
    c->nmin[a] = norm_min[a];
    c->nmax[a] = norm_max[a];
  }
  c->n_poses = 0;  // per-pose state depends on the skeleton
  c->sub_pose = -1;
  c->box_pose = -1;
  c->blist_pose = -1;
  c->sub_all_valid = false;
  c->tblist_valid = false;
  c->have_occ = false;
  c->fwd_valid = false;
  return IA_OK;
}

ia_status ia_param_sizes(const ia_ctx* c, int64_t* table_floats, int64_t* mlp_floats) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (table_floats) *table_floats = c->n_entries * 2;
  if (mlp_floats) *mlp_floats = (int64_t)kWidth * c->n_in + kWidth + kWidth * kWidth + kWidth + 4 * kWidth + 4;
  return IA_OK;
}

ia_status ia_set_params(ia_ctx* c, const float* table, const float* mlp, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!table || !mlp) return fail(c, IA_ERR_ARG, "null argument");
  int64_t nt = 0, nm = 0;
  ia_param_sizes(c, &nt, &nm);
  cudaStream_t s = (cudaStream_t)stream;
  IA_CUDA(c, cudaMemcpyAsync(c->d_table, table, sizeof(float) * nt, cudaMemcpyDefault, s), "ia_set_params");
  IA_CUDA(c, cudaMemcpyAsync(c->d_mlp, mlp, sizeof(float) * nm, cudaMemcpyDefault, s), "ia_set_params");
  if (c->d_table_h) IA_CUDA(c, launch_table_to_half(c->d_table, c->d_table_h, c->n_entries, s), "ia_set_params");
  if (c->fwd_own_params) c->fwd_valid = false;
  if (c->d_fm) {  // new parameters: the Adam state restarts
    dfree(c->d_fm);
    dfree(c->d_fv);
    c->field_step = 0;
  }
  c->have_params = true;
  return IA_OK;
}

ia_status ia_get_params(ia_ctx* c, float* table, float* mlp, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!c->have_params) return fail(c, IA_ERR_STATE, "ia_set_params has not been called");
  int64_t nt = 0, nm = 0;
  ia_param_sizes(c, &nt, &nm);
  cudaStream_t s = (cudaStream_t)stream;
  if (table) IA_CUDA(c, cudaMemcpyAsync(table, c->d_table, sizeof(float) * nt, cudaMemcpyDefault, s), "ia_get_params");
  if (mlp) IA_CUDA(c, cudaMemcpyAsync(mlp, c->d_mlp, sizeof(float) * nm, cudaMemcpyDefault, s), "ia_get_params");
  IA_CUDA(c, cudaStreamSynchronize(s), "ia_get_params");
  return IA_OK;
}

ia_status ia_set_pose(ia_ctx* c, int n_poses, const double* axis_angle, const double* root_trans, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (c->nb == 0) return fail(c, IA_ERR_STATE, "ia_set_skeleton has not been called");
  if (n_poses < 1 || n_poses > 4096) return fail(c, IA_ERR_ARG, "n_poses must be 1..4096");
  if (!axis_angle || !root_trans) return fail(c, IA_ERR_ARG, "null argument");
  const size_t nth = (size_t)n_poses * c->nb * 3;
  for (size_t i = 0; i < nth; ++i)
    if (!std::isfinite(axis_angle[i])) return fail(c, IA_ERR_ARG, "axis_angle must be finite");
  for (int i = 0; i < 3 * n_poses; ++i)
    if (!std::isfinite(root_trans[i])) return fail(c, IA_ERR_ARG, "root_trans must be finite");
  const size_t V = (size_t)c->Rw * c->Rw * c->Rw;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_poses > c->pose_cap) {
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_set_pose");
    c->pose_cap = 0;
    IA_CUDA(c, dalloc(&c->d_N, (size_t)n_poses * c->nb * 12), "ia_set_pose");
    IA_CUDA(c, dalloc(&c->d_Ninv, (size_t)n_poses * c->nb * 12), "ia_set_pose");
    IA_CUDA(c, dalloc(&c->d_B0inv, (size_t)n_poses * 12), "ia_set_pose");
    IA_CUDA(c, dalloc(&c->d_M, (size_t)n_poses * V * 3), "ia_set_pose");
    IA_CUDA(c, dalloc(&c->d_theta, nth), "ia_set_pose");
    IA_CUDA(c, dalloc(&c->d_trans, (size_t)n_poses * 3), "ia_set_pose");
    c->pose_cap = n_poses;
  }
  IA_CUDA(c, cudaMemcpyAsync(c->d_theta, axis_angle, sizeof(double) * nth, cudaMemcpyHostToDevice, s), "ia_set_pose");
  IA_CUDA(c, cudaMemcpyAsync(c->d_trans, root_trans, sizeof(double) * 3 * n_poses, cudaMemcpyHostToDevice, s),
          "ia_set_pose");
  IA_CUDA(c, launch_pose_chain(n_poses, c->nb, c->d_parent, c->d_rest, c->d_theta, c->d_trans, c->d_N, c->d_Ninv,
                               c->d_B0inv, s),
          "ia_set_pose: pose chain");
  c->sub_pose = -1;  // the culling masks belong to the previous grids
  c->box_pose = -1;
  c->blist_pose = -1;
  c->sub_all_valid = false;
  c->tblist_valid = false;
  c->fwd_valid = false;
  IA_CUDA(c, launch_blend(n_poses, (int)V, c->nb, c->d_skin, c->d_N, c->d_M, s), "ia_set_pose: blend grid");
  c->n_poses = n_poses;
  return IA_OK;
}

ia_status ia_get_transforms(ia_ctx* c, int pose, float* N, float* Ninv, float* B0inv, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (c->n_poses == 0) return fail(c, IA_ERR_STATE, "ia_set_pose has not been called");
  if (pose < 0 || pose >= c->n_poses) return fail(c, IA_ERR_ARG, "pose out of range");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)c->nb * 12;
  if (N) IA_CUDA(c, cudaMemcpyAsync(N, c->d_N + pose * n, n * 4, cudaMemcpyDefault, s), "ia_get_transforms");
  if (Ninv) IA_CUDA(c, cudaMemcpyAsync(Ninv, c->d_Ninv + pose * n, n * 4, cudaMemcpyDefault, s), "ia_get_transforms");
  if (B0inv)
    IA_CUDA(c, cudaMemcpyAsync(B0inv, c->d_B0inv + pose * 12, 48, cudaMemcpyDefault, s), "ia_get_transforms");
  IA_CUDA(c, cudaStreamSynchronize(s), "ia_get_transforms");
  return IA_OK;
}

ia_status ia_update_occupancy(ia_ctx* c, int pose, int mode, float* sigma_out, uint32_t* bits_out,
                              ia_render_stats* stats, void* stream) {
  ia_status st = need_ready(c, pose, false);
  if (st != IA_OK) return st;
  if (mode != IA_OCC_POSE && mode != IA_OCC_UNION) return fail(c, IA_ERR_ARG, "unknown occupancy mode %d", mode);
  cudaStream_t s = (cudaStream_t)stream;
  const int R = c->cfg.occ_res;
  const size_t words = ((size_t)R * R * R + 31) / 32;
  float* sig = sigma_out ? sigma_out : c->d_sigma;
  IA_CUDA(c, cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, s), "ia_update_occupancy");
  IA_CUDA(c, occ_density(c, pose, nullptr, sig, c->d_stats, s, false), "ia_update_occupancy: density");
  if (mode == IA_OCC_POSE) {
    IA_CUDA(c, launch_occ_bits(sig, R, c->cfg.occ_dilate, c->cfg.occ_tau, c->d_occ, nullptr, s),
            "ia_update_occupancy: bits");
    c->have_occ = true;
    IA_CUDA(c, rebuild_box_lists(c, s), "ia_update_occupancy: box lists");
    if (bits_out)
      IA_CUDA(c, cudaMemcpyAsync(bits_out, c->d_occ, words * 4, cudaMemcpyDeviceToDevice, s), "ia_update_occupancy");
  } else {
    IA_CUDA(c, launch_occ_bits(sig, R, c->cfg.occ_dilate, c->cfg.occ_tau, bits_out, c->d_occ_train, s),
            "ia_update_occupancy: union");
  }
  if (stats) read_stats(c, stats, s);
  return IA_OK;
}

ia_status ia_update_occupancy_ema(ia_ctx* c, int pose, const float* jitter, float decay, float* density_out,
                                  uint32_t* bits_out, ia_render_stats* stats, void* stream) {
  ia_status st = need_ready(c, pose, false);
  if (st != IA_OK) return st;
  if (!(decay >= 0.f && decay <= 1.f)) return fail(c, IA_ERR_ARG, "decay must be in [0, 1]");
  if (jitter && !is_device_ptr(jitter)) return fail(c, IA_ERR_ARG, "jitter must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  const int R = c->cfg.occ_res, n = R * R * R;
  const size_t words = ((size_t)n + 31) / 32;
  IA_CUDA(c, cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, s), "ia_update_occupancy_ema");
  IA_CUDA(c, occ_density(c, pose, jitter, c->d_sigma, c->d_stats, s, false), "ia_update_occupancy_ema: density");
  IA_CUDA(c, launch_occ_ema(c->d_sigma, c->d_occ_ema, n, decay, s), "ia_update_occupancy_ema: running density");
  IA_CUDA(c, launch_occ_bits(c->d_occ_ema, R, c->cfg.occ_dilate, c->cfg.occ_tau, c->d_occ_train, nullptr, s),
          "ia_update_occupancy_ema: bits");
  if (bits_out)
    IA_CUDA(c, cudaMemcpyAsync(bits_out, c->d_occ_train, words * 4, cudaMemcpyDeviceToDevice, s),
            "ia_update_occupancy_ema");
  if (density_out)
    IA_CUDA(c, cudaMemcpyAsync(density_out, c->d_occ_ema, sizeof(float) * n, cudaMemcpyDeviceToDevice, s),
            "ia_update_occupancy_ema");
  if (stats) read_stats(c, stats, s);
  return IA_OK;
}

ia_status ia_occupancy_from_density(ia_ctx* c, const float* sigma, uint32_t* bits_out, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!sigma) return fail(c, IA_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int R = c->cfg.occ_res;
  const size_t words = ((size_t)R * R * R + 31) / 32;
  IA_CUDA(c, launch_occ_bits(sigma, R, c->cfg.occ_dilate, c->cfg.occ_tau, c->d_occ, nullptr, s),
          "ia_occupancy_from_density");
  c->have_occ = true;
  IA_CUDA(c, rebuild_box_lists(c, s), "ia_occupancy_from_density: box lists");
  if (bits_out)
    IA_CUDA(c, cudaMemcpyAsync(bits_out, c->d_occ, words * 4, cudaMemcpyDeviceToDevice, s), "ia_occupancy_from_density");
  return IA_OK;
}

ia_status ia_set_occupancy(ia_ctx* c, const uint32_t* bits, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!bits) return fail(c, IA_ERR_ARG, "null argument");
  const int R = c->cfg.occ_res;
  const size_t words = ((size_t)R * R * R + 31) / 32;
  IA_CUDA(c, cudaMemcpyAsync(c->d_occ, bits, words * 4, cudaMemcpyDefault, (cudaStream_t)stream), "ia_set_occupancy");
  c->have_occ = true;
  IA_CUDA(c, rebuild_box_lists(c, (cudaStream_t)stream), "ia_set_occupancy: box lists");
  return IA_OK;
}

ia_status ia_query_posed(ia_ctx* c, int pose, int n, const float* x, float* sigma, float* rgb, float* x_canon,
                         int32_t* start, void* stream) {
  ia_status st = need_ready(c, pose, false);
  if (st != IA_OK) return st;
  if (n < 0 || (n > 0 && !x)) return fail(c, IA_ERR_ARG, "bad point array");
  if (n == 0) return IA_OK;
  IA_CUDA(c, launch_query_posed(posed_args(c, pose), n, x, sigma, rgb, x_canon, start, (cudaStream_t)stream),
          "ia_query_posed");
  return IA_OK;
}

ia_status ia_query_canonical(ia_ctx* c, int n, const float* x, float* sigma, float* rgb, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (c->nb == 0) return fail(c, IA_ERR_STATE, "ia_set_skeleton has not been called");
  if (!c->have_params) return fail(c, IA_ERR_STATE, "ia_set_params has not been called");
  if (n < 0 || (n > 0 && (!x || !sigma || !rgb))) return fail(c, IA_ERR_ARG, "bad arrays");
  if (n == 0) return IA_OK;
  PosedArgs a = posed_args_params(c);
  IA_CUDA(c, launch_query_canonical(a, n, x, sigma, rgb, (cudaStream_t)stream), "ia_query_canonical");
  return IA_OK;
}

static ia_status check_camera(ia_ctx* c, const ia_camera* cam) {
  if (!cam) return fail(c, IA_ERR_ARG, "null camera");
  if (cam->width < 1 || cam->height < 1 || (int64_t)cam->width * cam->height > (1LL << 28))
    return fail(c, IA_ERR_ARG, "image size out of range");
  if (!(cam->fx != 0.f) || !(cam->fy != 0.f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy) ||
      !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
    return fail(c, IA_ERR_ARG, "bad intrinsics");
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(cam->c2w[i])) return fail(c, IA_ERR_ARG, "c2w must be finite");
  return IA_OK;
}

static RenderArgs render_args(ia_ctx* c, int pose, const ia_camera* cam) {
  RenderArgs a{};
  a.P = posed_args(c, pose);
  a.B0inv = c->d_B0inv + (size_t)pose * 12;
  a.occ = c->d_occ;
  a.sub = (c->occ_cull && c->sub_pose == pose) ? c->d_sub : nullptr;
  a.box = box_dev(c);
  a.cam.fx = cam->fx;
  a.cam.fy = cam->fy;
  a.cam.cx = cam->cx;
  a.cam.cy = cam->cy;
  a.cam.width = cam->width;
  a.cam.height = cam->height;
  for (int i = 0; i < 12; ++i) a.cam.c2w[i] = cam->c2w[i];
  a.n_slots = c->cfg.max_samples;
  a.early_T = c->cfg.early_stop_T;
  a.tiles_x = (cam->width + kTile - 1) / kTile;
  const int tiles_y = (cam->height + kTile - 1) / kTile;
  a.n_ray_ids = a.tiles_x * tiles_y * kTile * kTile;
  a.counter = c->d_counter;
  a.stats = c->d_stats;
  return a;
}

ia_status ia_march_mask(ia_ctx* c, int pose, const ia_camera* cam, uint32_t* slot_mask, void* stream) {
  ia_status st = need_ready(c, pose, true);
  if (st != IA_OK) return st;
  if ((st = check_camera(c, cam)) != IA_OK) return st;
  if (!slot_mask) return fail(c, IA_ERR_ARG, "null argument");
  IA_CUDA(c, launch_march_mask(render_args(c, pose, cam), slot_mask, (cudaStream_t)stream), "ia_march_mask");
  return IA_OK;
}

// The wavefront path: march (kept samples written per ray), the sample count
// read back (the per-sample arrays are sized from it; a frame that outgrows
// them grows them and is marched again), then the search and field kernels
// over chunks of at most kWfChunk samples (their item arrays are sized for
// one chunk), then compositing.
constexpr size_t kWfChunk = size_t(1) << 21;

static ia_status render_wavefront(ia_ctx* c, int pose, RenderArgs& a, size_t npix, cudaStream_t s) {
  ia_status st = IA_OK;
  const bool prop = a.P.search != 0;
  const int nb = c->nb;
  const int per0 = prop ? std::min(c->pcfg.top_k, nb) : nb;
  if (c->wf_ray_cap < npix || !c->d_wf_counts) {
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_render");
    c->wf_ray_cap = 0;
    IA_CUDA(c, dalloc(&c->d_wf_first, npix), "ia_render: wavefront arrays");
    IA_CUDA(c, dalloc(&c->d_wf_cnt, npix), "ia_render: wavefront arrays");
    IA_CUDA(c, dalloc(&c->d_wf_dt, npix), "ia_render: wavefront arrays");
    if (!c->d_wf_counts) IA_CUDA(c, dalloc(&c->d_wf_counts, (size_t)2), "ia_render: wavefront arrays");
    c->wf_ray_cap = npix;
  }
  WfArgs w{};
  w.n_samples = c->d_wf_counts;
  w.n_fb = c->d_wf_counts + 1;
  w.role = kWfRender;
  w.ray_first = c->d_wf_first;
  w.ray_cnt = c->d_wf_cnt;
  w.ray_dt = c->d_wf_dt;
  unsigned n_host = 0;
  bool fits = false;
  for (int attempt = 0; attempt < 2 && !fits; ++attempt) {
    if (attempt > 0) {
      // the frame outgrew the sample arrays: grow them (with some room) and march again
      const size_t cap = (size_t)n_host + n_host / 4 + 1024;
      if (cap > (size_t)INT32_MAX / 2) return fail(c, IA_ERR_ARG, "ia_render: too many samples in the frame");
      IA_CUDA(c, cudaStreamSynchronize(s), "ia_render");
      c->wf_cap = 0;
      IA_CUDA(c, dalloc(&c->d_wf_xn, cap), "ia_render: wavefront arrays");
      IA_CUDA(c, dalloc(&c->d_wf_res, cap), "ia_render: wavefront arrays");
      c->wf_cap = cap;
      IA_CUDA(c, cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, s), "ia_render");
    }
    w.cap = (int)c->wf_cap;
    w.xn = c->d_wf_xn;
    IA_CUDA(c, cudaMemsetAsync(c->d_wf_counts, 0, 2 * sizeof(unsigned), s), "ia_render");
    IA_CUDA(c, launch_wf_march(a, w, s), "ia_render: march");
    IA_CUDA(c, cudaMemcpyAsync(&n_host, c->d_wf_counts, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "ia_render");
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_render");
    fits = n_host <= c->wf_cap;
  }
  if (!fits) return fail(c, IA_ERR_STATE, "ia_render: the frame's sample count changed between marches");
  // the chunk's arrays, sized for min(samples, kWfChunk) and the search mode
  const size_t chunk = std::min<size_t>(n_host, kWfChunk);
  if ((st = ensure_wf_items(c, chunk, per0, prop, s)) != IA_OK) return st;
  w.cap = (int)c->wf_cap;
  w.xn = c->d_wf_xn;
  w.res = c->d_wf_res;
  w.pose_stride = 0;  // one pose
  w.ninv = a.P.Ninv;
  w.n_ninv = nb * 12;
  w.prop = c->d_wf_prop;
  w.item0 = c->d_wf_item0;
  w.item1 = c->d_wf_item1;
  w.fb = c->d_wf_fb;
  w.fbidx = c->d_wf_fbidx;
  if (prop && c->occ_cull && c->sub_pose == pose && c->blist_pose == pose) {
    w.blist_count = c->d_blist_count;
    w.blist = c->d_blist;
    w.blist_cap = kBoxListCap;
    w.blist_scan = kBoxListCap;  // the render's lists hold occupied cells only: scan them whole
    w.cell_box = c->d_cell_box;
    w.blist_pose_cells = 0;  // one pose (the samples' pose bits are 0)
    w.box_pose_cells = 0;
  }
  for (size_t s0 = 0; s0 < n_host; s0 += chunk) {
    w.s0 = (int)s0;
    w.ns = (int)std::min(chunk, (size_t)n_host - s0);
    IA_CUDA(c, launch_wf_chunk(a, w, c->num_sms, s), "ia_render: kernels");
  }
  IA_CUDA(c, launch_wf_composite(a, w, s), "ia_render: compositing");
  return IA_OK;
}

ia_status ia_set_render_path(ia_ctx* c, int path) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (path != IA_RENDER_FUSED && path != IA_RENDER_WAVEFRONT) return fail(c, IA_ERR_ARG, "unknown render path");
  c->render_path = path;
  return IA_OK;
}

ia_status ia_render(ia_ctx* c, int pose, const ia_camera* cam, float* rgb, float* alpha, ia_render_stats* stats,
                    void* stream) {
  ia_status st = need_ready(c, pose, true);
  if (st != IA_OK) return st;
  if ((st = check_camera(c, cam)) != IA_OK) return st;
  if (!rgb || !alpha) return fail(c, IA_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t npix = (size_t)cam->width * cam->height;
  const bool dev_rgb = is_device_ptr(rgb), dev_alpha = is_device_ptr(alpha);
  float* o_rgb = rgb;
  float* o_alpha = alpha;
  if (!dev_rgb || !dev_alpha) {
    if (c->out_cap < npix * 4) {
      IA_CUDA(c, cudaStreamSynchronize(s), "ia_render");
      c->out_cap = 0;
      IA_CUDA(c, dalloc(&c->d_out, npix * 4), "ia_render: output scratch");
      c->out_cap = npix * 4;
    }
    if (!dev_rgb) o_rgb = c->d_out;
    if (!dev_alpha) o_alpha = c->d_out + 3 * npix;
  }
  RenderArgs a = render_args(c, pose, cam);
  a.rgb = o_rgb;
  a.alpha = o_alpha;
  IA_CUDA(c, cudaMemsetAsync(c->d_stats, 0, sizeof(unsigned long long) * ST_COUNT, s), "ia_render");
  if (c->render_path == IA_RENDER_WAVEFRONT) {
    st = render_wavefront(c, pose, a, npix, s);
    if (st != IA_OK) return st;
  } else {
    IA_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned int), s), "ia_render");
    IA_CUDA(c, launch_render(a, c->num_sms, s), "ia_render: kernel");
  }
  if (!dev_rgb) IA_CUDA(c, cudaMemcpyAsync(rgb, o_rgb, npix * 12, cudaMemcpyDeviceToHost, s), "ia_render: copy");
  if (!dev_alpha) IA_CUDA(c, cudaMemcpyAsync(alpha, o_alpha, npix * 4, cudaMemcpyDeviceToHost, s), "ia_render: copy");
  if (!dev_rgb || !dev_alpha) IA_CUDA(c, cudaStreamSynchronize(s), "ia_render");
  if (stats) read_stats(c, stats, s);
  return IA_OK;
}

namespace {

// Checks and workspace shared by the training calls, and the arguments of their
// kernels (parameters, poses, grid, batch and workspace; no gradient buffers).
// need_target: the step computes its own loss from the batch's targets.
ia_status train_prepare(ia_ctx* c, const ia_batch* b, int occ_grid, bool need_target, cudaStream_t s,
                        TrainArgs& a) {
  ia_status st = need_ready(c, 0, false);
  if (st != IA_OK) return st;
  if (!b) return fail(c, IA_ERR_ARG, "null argument");
  if (b->n_rays < 1 || b->n_rays > (1 << 24)) return fail(c, IA_ERR_ARG, "n_rays must be 1..2^24");
  if (!b->origin || !b->direction || !b->pose || (need_target && !b->target))
    return fail(c, IA_ERR_ARG, "null batch array");
  if (occ_grid != IA_OCC_POSE && occ_grid != IA_OCC_UNION) return fail(c, IA_ERR_ARG, "unknown occupancy grid");
  if (occ_grid == IA_OCC_POSE && !c->have_occ) return fail(c, IA_ERR_STATE, "no render grid (ia_update_occupancy)");
  if (b->n_reg < 0 || b->n_reg > (1 << 24)) return fail(c, IA_ERR_ARG, "n_reg must be 0..2^24");
  if (b->n_reg > 0 && (!b->reg_x || !b->reg_pose)) return fail(c, IA_ERR_ARG, "null regulariser array");
  if (b->n_reg > 0 && !(std::isfinite(b->reg_weight))) return fail(c, IA_ERR_ARG, "reg_weight must be finite");
  if (need_target && c->loss.w_alpha != 0.f && !b->alpha_target)
    return fail(c, IA_ERR_ARG, "the loss has an alpha term: batch->alpha_target is needed");
  const int n = b->n_rays, N = c->cfg.max_samples;
  const size_t cap = (size_t)n * N + (size_t)b->n_reg;
  if (n > c->ray_cap || cap > c->s_cap) {
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_train_step");
    c->ray_cap = 0;
    c->s_cap = 0;
    IA_CUDA(c, dalloc(&c->d_ray_n, (size_t)n), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_ray_dt, (size_t)n), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_ray_idx, (size_t)n * N), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_count, (size_t)1), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_s_pos, cap), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_s_out, cap), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_s_x, cap), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_s_grad, cap), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_s_dfeat, cap * (kIn / 4)), "ia_train_step: workspace");
    IA_CUDA(c, dalloc(&c->d_s_gx, cap), "ia_train_step: workspace");
    if (c->cfg.precision == IA_FP32) {
      IA_CUDA(c, dalloc(&c->d_act, cap * kActStride), "ia_train_step: workspace");
    } else {
      // rows that the backward never writes must stay zero: clear once here
      const int64_t ld = ((int64_t)cap + kWgChunk - 1) / kWgChunk * kWgChunk;
      IA_CUDA(c, dalloc(&c->d_X, (size_t)kWgRows * ld), "ia_train_step: workspace");
      IA_CUDA(c, cudaMemset(c->d_X, 0, sizeof(uint16_t) * kWgRows * ld), "ia_train_step: workspace");
      IA_CUDA(c, make_wgrad_map(&c->x_map, c->d_X, ld, c->cfg.precision == IA_BF16), "ia_train_step: tensor map");
      c->x_ld = ld;
    }
    c->ray_cap = n;
    c->s_cap = cap;
  }
  if (b->n_reg > c->reg_cap) {
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_train_step");
    c->reg_cap = 0;
    IA_CUDA(c, dalloc(&c->d_reg_idx, (size_t)b->n_reg), "ia_train_step: workspace");
    c->reg_cap = b->n_reg;
  }
  if (c->cfg.precision != IA_FP32 && !c->d_scale) {
    IA_CUDA(c, dalloc(&c->d_scale, (size_t)1), "ia_train_step: loss scale");
    IA_CUDA(c, dalloc(&c->d_overflow, (size_t)1), "ia_train_step: loss scale");
    IA_CUDA(c, dalloc(&c->d_good, (size_t)1), "ia_train_step: loss scale");
    const float s0 = c->cfg.precision == IA_FP16 ? kInitialLossScale : 1.f;
    IA_CUDA(c, cudaMemcpy(c->d_scale, &s0, sizeof(float), cudaMemcpyHostToDevice), "ia_train_step: loss scale");
    IA_CUDA(c, cudaMemset(c->d_good, 0, sizeof(int)), "ia_train_step: loss scale");
  }
  const size_t V = (size_t)c->Rw * c->Rw * c->Rw;
  IA_CUDA(c, cudaMemsetAsync(c->d_count, 0, sizeof(int), s), "ia_train_step");
  IA_CUDA(c, cudaMemsetAsync(c->d_tstats, 0, sizeof(unsigned long long) * ST_COUNT, s), "ia_train_step");
  IA_CUDA(c, cudaMemsetAsync(c->d_work + 1, 0, sizeof(unsigned), s), "ia_train_step");
  if (c->n_poses > c->pose_ws_cap) {
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_train_step");
    c->pose_ws_cap = 0;
    IA_CUDA(c, dalloc(&c->d_pose_ws, (size_t)2 * c->n_poses), "ia_train_step: workspace");
    c->pose_ws_cap = c->n_poses;
  }
  IA_CUDA(c, cudaMemsetAsync(c->d_pose_ws, 0, sizeof(int) * 2 * c->n_poses, s), "ia_train_step");
  a = TrainArgs{};
  a.P = posed_args(c, 0);
  a.V = (int)V;
  a.box = box_dev(c);
  // root-culling masks of every pose, built on the first step after the blended
  // grids changed (one launch over all poses; skipped above 4 GiB)
  a.sub = nullptr;
  if (c->occ_cull) {
    const size_t per = (size_t)c->cfg.occ_res * c->cfg.occ_res * c->cfg.occ_res;
    if ((size_t)c->n_poses * per * sizeof(unsigned long long) <= (size_t(4) << 30)) {
      if (c->n_poses > c->sub_all_cap) {
        IA_CUDA(c, cudaStreamSynchronize(s), "ia_train_step");
        c->sub_all_cap = 0;
        c->sub_all_valid = false;
        c->tblist_valid = false;
        IA_CUDA(c, dalloc(&c->d_sub_all, (size_t)c->n_poses * per), "ia_train_step: culling masks");
        c->sub_all_cap = c->n_poses;
      }
      // the fallback point test's boxes and lists, with the proposal search
      const bool lists = a.P.search != 0 && (size_t)c->n_poses * per * kBoxListCap * sizeof(int) <= (size_t(4) << 30);
      const int nc = c->Rw - 1;
      if (lists && c->n_poses > c->tblist_cap) {
        IA_CUDA(c, cudaStreamSynchronize(s), "ia_train_step");
        c->tblist_cap = 0;
        c->tblist_valid = false;
        IA_CUDA(c, dalloc(&c->d_tcell_box, (size_t)c->n_poses * 2 * nc * nc * nc), "ia_train_step: culling boxes");
        IA_CUDA(c, dalloc(&c->d_tblist_count, (size_t)c->n_poses * per), "ia_train_step: culling boxes");
        IA_CUDA(c, dalloc(&c->d_tblist, (size_t)c->n_poses * per * kBoxListCap), "ia_train_step: culling boxes");
        c->tblist_cap = c->n_poses;
      }
      if (!c->sub_all_valid || (lists && !c->tblist_valid)) {
        IA_CUDA(c, launch_occ_cover(a.P.S, (int)V, c->n_poses, a.P.cfg, a.box, c->d_sub_all, nullptr, s,
                                    lists ? c->d_tcell_box : nullptr),
                "ia_train_step: culling masks");
        c->sub_all_valid = true;
        c->tblist_valid = false;
        if (lists) {
          IA_CUDA(c, launch_occ_boxlist(c->d_tcell_box, nc * nc * nc, c->n_poses, a.box, nullptr, c->d_tblist_count,
                                        c->d_tblist, kBoxListCap, s),
                  "ia_train_step: culling box lists");
          c->tblist_valid = true;
        }
      }
      a.sub = c->d_sub_all;
    }
  }
  a.B0inv = c->d_B0inv;
  a.N = c->d_N;
  a.skin = c->d_skin;
  a.occ = occ_grid == IA_OCC_POSE ? c->d_occ : c->d_occ_train;
  a.n_slots = N;
  a.n_rays = n;
  a.origin = b->origin;
  a.direction = b->direction;
  a.pose = b->pose;
  a.n_poses = c->n_poses;
  a.target = b->target;
  a.count = c->d_count;
  a.ray_n = c->d_ray_n;
  a.ray_dt = c->d_ray_dt;
  a.ray_idx = c->d_ray_idx;
  a.s_pos = c->d_s_pos;
  a.s_out = c->d_s_out;
  a.s_x = c->d_s_x;
  a.s_grad = c->d_s_grad;
  a.s_dfeat = c->d_s_dfeat;
  a.s_gx = c->d_s_gx;
  a.work = c->d_work + 1;
  a.n_reg = b->n_reg;
  a.reg_x = b->reg_x;
  a.reg_pose = b->reg_pose;
  a.reg_weight = b->reg_weight;
  a.reg_idx = c->d_reg_idx;
  a.huber = c->loss.rgb_loss == IA_LOSS_HUBER ? 1 : 0;
  a.huber_delta = c->loss.huber_delta;
  a.w_rgb = c->loss.w_rgb;
  a.w_alpha = c->loss.w_alpha;
  a.w_hard = c->loss.w_hard;
  a.alpha_target = b->alpha_target;
  a.act = c->d_act;
  a.act_ld = (int64_t)c->s_cap;
  a.prec = c->cfg.precision;
  a.X = c->d_X;
  a.ld = c->x_ld;
  a.scale = c->d_scale;
  a.overflow = c->d_overflow;
  a.good_steps = c->d_good;
  a.wait_ns = c->wait_ns;
  a.inject = c->inject;
  a.theta_all = c->d_theta;
  a.stats = c->d_tstats;
  a.pose_tot = c->d_pose_ws;
  a.pose_fill = c->d_pose_ws + c->n_poses;
  // the forward's search and field: the wavefront kernels over the emitted
  // samples, one chunk whose size the device holds
  {
    const bool wprop = a.P.search != 0 && c->cfg.precision != IA_FP32;
    const int per0 = wprop ? std::min(c->pcfg.top_k, c->nb) : c->nb;
    ia_status st2 = ensure_wf_items(c, c->s_cap, per0, wprop, s);
    if (st2 != IA_OK) return st2;
    WfArgs& w = a.wf;
    w = WfArgs{};
    w.xn = c->d_s_pos;
    w.res = c->d_s_out;
    w.xs = c->d_s_x;
    w.cap = (int)c->s_cap;
    w.pose_stride = (int)(3 * V);
    w.ninv = a.P.Ninv;
    w.n_ninv = c->n_poses * c->nb * 12;
    w.s0 = 0;
    w.ns = (int)c->s_cap;
    w.ns_dev = reinterpret_cast<const unsigned*>(c->d_count);
    w.prop = c->d_wf_prop;
    w.item0 = c->d_wf_item0;
    w.item1 = c->d_wf_item1;
    w.fb = c->d_wf_fb;
    w.fbidx = c->d_wf_fbidx;
    w.n_fb = c->d_wf_counts + 1;
    w.role = kWfTrain;
    if (a.sub && a.P.search && c->tblist_valid) {
      w.blist_count = c->d_tblist_count;
      w.blist = c->d_tblist;
      w.blist_cap = kBoxListCap;
      w.blist_scan = 16;  // the training lists hold every cell a box meets: only short ones pay
      w.cell_box = c->d_tcell_box;
      w.blist_pose_cells = c->cfg.occ_res * c->cfg.occ_res * c->cfg.occ_res;
      w.box_pose_cells = (c->Rw - 1) * (c->Rw - 1) * (c->Rw - 1);
    }
  }
  if (a.P.search) {
    if (c->n_poses > c->pb1_cap) {
      IA_CUDA(c, cudaStreamSynchronize(s), "ia_train_step");
      c->pb1_cap = 0;
      IA_CUDA(c, dalloc(&c->d_pb1, (size_t)c->n_poses * kWidth), "ia_train_step: workspace");
      c->pb1_cap = c->n_poses;
    }
    a.P.prop.b1p = c->d_pb1;
  }
  return IA_OK;
}

// Gradient buffers of a backward: checked, zeroed (with the step's skip flags),
// and entered into the kernel arguments.
ia_status train_grads(ia_ctx* c, const ia_grads* g, cudaStream_t s, TrainArgs& a) {
  if (!g || !g->table || !g->mlp || !g->skin || !g->bones) return fail(c, IA_ERR_ARG, "null gradient buffer");
  if ((reinterpret_cast<uintptr_t>(g->table) & 7) != 0)
    return fail(c, IA_ERR_ARG, "grads->table must be 8-byte aligned (one float pair per entry)");
  int64_t nt = 0, nm = 0;
  ia_param_sizes(c, &nt, &nm);
  const size_t V = (size_t)c->Rw * c->Rw * c->Rw;
  if (c->d_overflow) IA_CUDA(c, cudaMemsetAsync(c->d_overflow, 0, sizeof(int), s), "ia_train_step");
  IA_CUDA(c, cudaMemsetAsync(g->table, 0, sizeof(float) * nt, s), "ia_train_step");
  IA_CUDA(c, cudaMemsetAsync(g->mlp, 0, sizeof(float) * nm, s), "ia_train_step");
  IA_CUDA(c, cudaMemsetAsync(g->skin, 0, sizeof(float) * V * c->nb, s), "ia_train_step");
  IA_CUDA(c, cudaMemsetAsync(g->bones, 0, sizeof(float) * c->n_poses * c->nb * 12, s), "ia_train_step");
  a.skin_vec = (c->nb % 4 == 0 && (reinterpret_cast<uintptr_t>(g->skin) & 15) == 0 &&
                (reinterpret_cast<uintptr_t>(c->d_skin) & 15) == 0) ? 1 : 0;
  a.g_table = g->table;
  a.g_mlp = g->mlp;
  a.g_skin = g->skin;
  a.g_bones = g->bones;
  a.n_table_f = (size_t)nt;
  a.n_mlp_f = (size_t)nm;
  a.n_skin_f = V * c->nb;
  a.n_bones_f = (size_t)c->n_poses * c->nb * 12;
  return IA_OK;
}

}  // namespace

ia_status ia_train_step(ia_ctx* c, const ia_batch* b, int occ_grid, float* loss, float* rgb_out,
                        const ia_grads* g, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!loss) return fail(c, IA_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  TrainArgs a;
  ia_status st = train_prepare(c, b, occ_grid, true, s, a);
  if (st != IA_OK) return st;
  if ((st = train_grads(c, g, s, a)) != IA_OK) return st;
  c->fwd_valid = false;  // the workspace is this step's now
  a.comp_mode = kCompLoss;
  a.loss = loss;
  a.rgb_out = rgb_out;
  IA_CUDA(c, launch_train(a, &c->x_map, c->num_sms, s), "ia_train_step: kernels");
  return IA_OK;
}

ia_status ia_train_forward(ia_ctx* c, const ia_batch* b, int occ_grid, const float* table, const float* mlp,
                           float* rgb_out, float* alpha_out, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!rgb_out) return fail(c, IA_ERR_ARG, "null rgb_out");
  if (b && b->n_reg != 0) return fail(c, IA_ERR_ARG, "the regulariser needs ia_train_step (n_reg must be 0)");
  if ((table && !is_device_ptr(table)) || (mlp && !is_device_ptr(mlp)) || !is_device_ptr(rgb_out) ||
      (alpha_out && !is_device_ptr(alpha_out)))
    return fail(c, IA_ERR_ARG, "table, mlp, rgb_out and alpha_out must be device memory");
  if (table && (reinterpret_cast<uintptr_t>(table) & 7) != 0)
    return fail(c, IA_ERR_ARG, "table must be 8-byte aligned (one float pair per entry)");
  cudaStream_t s = (cudaStream_t)stream;
  TrainArgs a;
  c->fwd_valid = false;
  ia_status st = train_prepare(c, b, occ_grid, false, s, a);
  if (st != IA_OK) return st;
  if (table) {
    a.P.F.table = reinterpret_cast<const float2*>(table);
    if (c->cfg.precision != IA_FP32) {
      if (!c->d_table_h_ext) IA_CUDA(c, dalloc(&c->d_table_h_ext, (size_t)c->n_entries), "ia_train_forward");
      IA_CUDA(c, launch_table_to_half(table, c->d_table_h_ext, c->n_entries, s), "ia_train_forward");
      a.P.table_h = c->d_table_h_ext;
    }
  }
  if (mlp) a.P.mlp = mlp;
  a.comp_mode = kCompForward;
  a.rgb_out = rgb_out;
  a.alpha_out = alpha_out;
  IA_CUDA(c, launch_train_forward(a, c->num_sms, s), "ia_train_forward: kernels");
  IA_CUDA(c, launch_train_composite(a, s), "ia_train_forward: compositing");
  c->fwd = a;
  c->fwd_valid = true;
  c->fwd_own_params = !table || !mlp;
  return IA_OK;
}

ia_status ia_train_backward(ia_ctx* c, const float* grad_rgb, const float* grad_alpha, const ia_grads* g,
                            void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!c->fwd_valid)
    return fail(c, IA_ERR_STATE, "no ia_train_forward to differentiate (or its state changed since)");
  if (!grad_rgb || !is_device_ptr(grad_rgb) || (grad_alpha && !is_device_ptr(grad_alpha)))
    return fail(c, IA_ERR_ARG, "grad_rgb (and grad_alpha) must be device memory");
  cudaStream_t s = (cudaStream_t)stream;
  TrainArgs a = c->fwd;
  ia_status st = train_grads(c, g, s, a);
  if (st != IA_OK) return st;
  a.comp_mode = kCompUpstream;
  a.up_rgb = grad_rgb;
  a.up_alpha = grad_alpha;
  a.rgb_out = nullptr;
  a.alpha_out = nullptr;
  a.loss = nullptr;
  a.wait_ns = c->wait_ns;
  a.inject = c->inject;
  IA_CUDA(c, launch_train_composite(a, s), "ia_train_backward: compositing");
  IA_CUDA(c, launch_train_backward(a, &c->x_map, c->num_sms, s), "ia_train_backward: kernels");
  return IA_OK;
}

ia_status ia_adam_step(ia_ctx* c, const float* g_table, const float* g_mlp, const float* g_skin, float lr,
                       float beta1, float beta2, float eps, void* stream) {
  if (!c || !g_table || !g_mlp) return fail(c, IA_ERR_ARG, "null argument");
  if (!c->have_params) return fail(c, IA_ERR_STATE, "ia_set_params has not been called");
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(c, IA_ERR_ARG, "bad Adam hyper-parameters");
  if (!is_device_ptr(g_table) || !is_device_ptr(g_mlp) || (g_skin && !is_device_ptr(g_skin)))
    return fail(c, IA_ERR_ARG, "gradients must be device memory");
  if (g_skin && c->nb == 0) return fail(c, IA_ERR_STATE, "ia_set_skeleton has not been called");
  cudaStream_t s = (cudaStream_t)stream;
  int64_t nt = 0, nm = 0;
  ia_param_sizes(c, &nt, &nm);
  if (!c->d_fm) {
    IA_CUDA(c, dalloc(&c->d_fm, (size_t)(nt + nm)), "ia_adam_step: moments");
    IA_CUDA(c, dalloc(&c->d_fv, (size_t)(nt + nm)), "ia_adam_step: moments");
    IA_CUDA(c, cudaMemsetAsync(c->d_fm, 0, sizeof(float) * (nt + nm), s), "ia_adam_step");
    IA_CUDA(c, cudaMemsetAsync(c->d_fv, 0, sizeof(float) * (nt + nm), s), "ia_adam_step");
    c->field_step = 0;
  }
  ++c->field_step;
  if (c->fwd_own_params) c->fwd_valid = false;
  // an overflowed reduced-precision step (zeroed gradients) leaves the state alone
  const int* skip = c->cfg.precision != IA_FP32 ? c->d_overflow : nullptr;
  IA_CUDA(c, launch_adam(c->d_table, g_table, c->d_fm, c->d_fv, nt, lr, c->field_step, beta1, beta2, eps, skip, s),
          "ia_adam_step: table");
  IA_CUDA(c, launch_adam(c->d_mlp, g_mlp, c->d_fm + nt, c->d_fv + nt, nm, lr, c->field_step, beta1, beta2, eps, skip,
                         s),
          "ia_adam_step: mlp");
  if (c->d_table_h) IA_CUDA(c, launch_table_to_half(c->d_table, c->d_table_h, c->n_entries, s), "ia_adam_step");
  if (g_skin) {
    // the learnable skinning-weight grid: its own moments, then every pose's blended grid again
    const size_t V = (size_t)c->Rw * c->Rw * c->Rw, ns = V * c->nb;
    if (!c->d_sm) {
      IA_CUDA(c, dalloc(&c->d_sm, ns), "ia_adam_step: moments");
      IA_CUDA(c, dalloc(&c->d_sv, ns), "ia_adam_step: moments");
      IA_CUDA(c, cudaMemsetAsync(c->d_sm, 0, sizeof(float) * ns, s), "ia_adam_step");
      IA_CUDA(c, cudaMemsetAsync(c->d_sv, 0, sizeof(float) * ns, s), "ia_adam_step");
      c->skin_step = 0;
    }
    ++c->skin_step;
    IA_CUDA(c, launch_adam(c->d_skin, g_skin, c->d_sm, c->d_sv, (int64_t)ns, lr, c->skin_step, beta1, beta2, eps, skip,
                           s),
            "ia_adam_step: skinning grid");
    // every culling mask depends on the skinning grid; the blended grids exist only once poses are set
    c->sub_pose = -1;
    c->box_pose = -1;
    c->blist_pose = -1;
    c->sub_all_valid = false;
    c->tblist_valid = false;
    c->fwd_valid = false;
    if (c->n_poses > 0) {
      IA_CUDA(c, launch_blend(c->n_poses, (int)V, c->nb, c->d_skin, c->d_N, c->d_M, s), "ia_adam_step: blend grid");
    }
  }
  return IA_OK;
}

ia_status ia_gather_probe(const float* table, int64_t n_records, int record_bytes, int iters, int blocks, float* sink,
                          void* stream) {
  if (!table || !sink || n_records < 1 || n_records > (1LL << 31) || iters < 1 || blocks < 1)
    return fail(nullptr, IA_ERR_ARG, "bad gather probe arguments");
  if (record_bytes != 4 && record_bytes != 8 && record_bytes != 16 && record_bytes != 48)
    return fail(nullptr, IA_ERR_ARG, "record_bytes must be 4, 8, 16 or 48");
  const uintptr_t align = record_bytes == 48 ? 16 : (uintptr_t)record_bytes;
  if ((reinterpret_cast<uintptr_t>(table) & (align - 1)) != 0)
    return fail(nullptr, IA_ERR_ARG, "table must be aligned to its records");
  cudaError_t e = launch_gather_probe(table, n_records, record_bytes, iters, blocks, sink, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "ia_gather_probe");
  return IA_OK;
}

ia_status ia_atomic_probe(float* table, int64_t n_records, int record_bytes, int iters, int blocks, void* stream) {
  if (!table || n_records < 1 || n_records > (1LL << 31) || iters < 1 || blocks < 1)
    return fail(nullptr, IA_ERR_ARG, "bad atomic probe arguments");
  if (record_bytes != 8 && record_bytes != 16) return fail(nullptr, IA_ERR_ARG, "record_bytes must be 8 or 16");
  if ((reinterpret_cast<uintptr_t>(table) & (uintptr_t)(record_bytes - 1)) != 0)
    return fail(nullptr, IA_ERR_ARG, "table must be aligned to its records");
  cudaError_t e = launch_atomic_probe(table, n_records, record_bytes, iters, blocks, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "ia_atomic_probe");
  return IA_OK;
}

ia_status ia_set_loss(ia_ctx* c, const ia_loss* l) {
  if (!c || !l) return fail(c, IA_ERR_ARG, "null argument");
  if (l->rgb_loss != IA_LOSS_L2 && l->rgb_loss != IA_LOSS_HUBER) return fail(c, IA_ERR_ARG, "unknown rgb_loss");
  if (l->rgb_loss == IA_LOSS_HUBER && !(l->huber_delta > 0.f && std::isfinite(l->huber_delta)))
    return fail(c, IA_ERR_ARG, "huber_delta must be positive");
  if (!std::isfinite(l->w_rgb) || !std::isfinite(l->w_alpha) || !std::isfinite(l->w_hard))
    return fail(c, IA_ERR_ARG, "loss weights must be finite");
  c->loss = *l;
  return IA_OK;
}

ia_status ia_grad_sizes(const ia_ctx* c, int64_t* skin_floats, int64_t* bone_floats) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (c->nb == 0) return fail(const_cast<ia_ctx*>(c), IA_ERR_STATE, "ia_set_skeleton has not been called");
  if (skin_floats) *skin_floats = (int64_t)c->Rw * c->Rw * c->Rw * c->nb;
  if (bone_floats) *bone_floats = (int64_t)c->n_poses * c->nb * 12;
  return IA_OK;
}

// IA_ERR_CUDA if the last reduced-precision step gave up waiting on its
// tensor-core pipeline (the step was skipped); waits on the stream
static ia_status pipeline_status(ia_ctx* c, cudaStream_t s, int* flags_out) {
  int flags = 0;
  if (c->d_overflow) {
    IA_CUDA(c, cudaMemcpyAsync(&flags, c->d_overflow, sizeof(int), cudaMemcpyDeviceToHost, s), "step flags");
    IA_CUDA(c, cudaStreamSynchronize(s), "step flags");
  }
  if (flags_out) *flags_out = flags;
  if (flags & kStepPipelineError)
    return fail(c, IA_ERR_CUDA,
                "the tensor-core weight-gradient reduction gave up waiting on its pipeline (the step was skipped)");
  return IA_OK;
}

ia_status ia_train_stats(ia_ctx* c, ia_render_stats* stats, void* stream) {
  if (!c || !stats) return fail(c, IA_ERR_ARG, "null argument");
  read_stats(c, stats, (cudaStream_t)stream, c->d_tstats);
  stats->early_stopped = 0;
  return pipeline_status(c, (cudaStream_t)stream, nullptr);
}

ia_status ia_set_wait_limit(ia_ctx* c, int64_t limit_ns) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (limit_ns < 0 || limit_ns > (int64_t)10000000000LL) return fail(c, IA_ERR_ARG, "limit_ns must be 0..1e10");
  c->wait_ns = limit_ns == 0 ? kDefaultWaitNs : (uint64_t)limit_ns;
  return IA_OK;
}

ia_status ia_set_fault_injection(ia_ctx* c, int flags) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (flags & ~IA_INJECT_WITHHOLD_COPY) return fail(c, IA_ERR_ARG, "unknown injection flag");
  c->inject = flags;
  return IA_OK;
}

ia_status ia_loss_scale(ia_ctx* c, float* scale, int32_t* skipped, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!scale && !skipped) return fail(c, IA_ERR_ARG, "null argument");
  if (!c->d_scale) {  // fp32, or no reduced-precision step yet
    if (scale) *scale = c->cfg.precision == IA_FP16 ? kInitialLossScale : 1.f;
    if (skipped) *skipped = 0;
    return IA_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (scale) IA_CUDA(c, cudaMemcpyAsync(scale, c->d_scale, sizeof(float), cudaMemcpyDeviceToHost, s), "ia_loss_scale");
  int flags = 0;
  const ia_status st = pipeline_status(c, s, &flags);
  if (skipped) *skipped = flags != 0 ? 1 : 0;
  if (st != IA_OK) return st;
  return IA_OK;
}

// ---------------------------------------------------------------------------
// Learned correspondence proposal
// ---------------------------------------------------------------------------

ia_status ia_proposal_init(ia_ctx* c, const ia_proposal_config* q) {
  if (!c || !q) return fail(c, IA_ERR_ARG, "null argument");
  if (c->nb == 0) return fail(c, IA_ERR_STATE, "ia_set_skeleton has not been called");
  if (q->n_levels < 1 || q->n_levels > 8) return fail(c, IA_ERR_ARG, "proposal n_levels must be 1..8");
  if (q->log2_table < 10 || q->log2_table > 24) return fail(c, IA_ERR_ARG, "proposal log2_table must be 10..24");
  for (int l = 0; l < q->n_levels; ++l)
    if (q->level_res[l] < 2 || q->level_res[l] > (1 << 16)) return fail(c, IA_ERR_ARG, "bad proposal level_res");
  if (q->top_k < 1 || q->top_k > 2) return fail(c, IA_ERR_ARG, "top_k must be 1 or 2");
  if (!(q->offset_weight >= 0.f) || !std::isfinite(q->offset_weight)) return fail(c, IA_ERR_ARG, "bad offset_weight");
  if (c->nb + 3 > kPropMaxOut) return fail(c, IA_ERR_LIMIT, "the proposal supports at most %d bones", kPropMaxOut - 3);
  const int64_t T = 1LL << q->log2_table;
  int64_t off = 0;
  for (int l = 0; l < q->n_levels; ++l) {
    const int64_t r1 = (int64_t)q->level_res[l] + 1, dense = r1 * r1 * r1;
    c->plv[l].res = q->level_res[l];
    c->plv[l].dense = dense <= T ? 1 : 0;
    c->plv[l].size = (uint32_t)(dense <= T ? dense : T);
    c->plv[l].offset = (uint32_t)off;
    off += c->plv[l].size;
  }
  c->pcfg = *q;
  c->p_entries = off;
  const int nin = 2 * q->n_levels + 3 * c->nb;
  c->p_mlp = (int64_t)kWidth * nin + kWidth + 2 * ((int64_t)kWidth * kWidth + kWidth) + (int64_t)(c->nb + 3) * kWidth +
             (c->nb + 3);
  const size_t np = (size_t)(2 * off + c->p_mlp);
  c->prop_ready = false;
  IA_CUDA(c, dalloc(&c->d_pp, np), "ia_proposal_init");
  c->d_ptable = c->d_pp;
  c->d_pmlp = c->d_pp + 2 * off;
  IA_CUDA(c, dalloc(&c->d_ploss, (size_t)1), "ia_proposal_init");
  IA_CUDA(c, dalloc(&c->d_pg, np), "ia_proposal_init");
  IA_CUDA(c, dalloc(&c->d_pm, np), "ia_proposal_init");
  IA_CUDA(c, dalloc(&c->d_pv, np), "ia_proposal_init");
  IA_CUDA(c, cudaMemset(c->d_ptable, 0, sizeof(float) * 2 * off), "ia_proposal_init");
  IA_CUDA(c, cudaMemset(c->d_pmlp, 0, sizeof(float) * c->p_mlp), "ia_proposal_init");
  IA_CUDA(c, cudaMemset(c->d_pm, 0, sizeof(float) * np), "ia_proposal_init");
  IA_CUDA(c, cudaMemset(c->d_pv, 0, sizeof(float) * np), "ia_proposal_init");
  c->adam_step = 0;
  c->prop_ready = true;
  return IA_OK;
}

ia_status ia_proposal_param_sizes(const ia_ctx* c, int64_t* table_floats, int64_t* mlp_floats) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!c->prop_ready) return fail(const_cast<ia_ctx*>(c), IA_ERR_STATE, "ia_proposal_init has not been called");
  if (table_floats) *table_floats = 2 * c->p_entries;
  if (mlp_floats) *mlp_floats = c->p_mlp;
  return IA_OK;
}

ia_status ia_proposal_set_params(ia_ctx* c, const float* table, const float* mlp, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!c->prop_ready) return fail(c, IA_ERR_STATE, "ia_proposal_init has not been called");
  if (!table || !mlp) return fail(c, IA_ERR_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t np = (size_t)(2 * c->p_entries + c->p_mlp);
  IA_CUDA(c, cudaMemcpyAsync(c->d_ptable, table, sizeof(float) * 2 * c->p_entries, cudaMemcpyDefault, s),
          "ia_proposal_set_params");
  IA_CUDA(c, cudaMemcpyAsync(c->d_pmlp, mlp, sizeof(float) * c->p_mlp, cudaMemcpyDefault, s), "ia_proposal_set_params");
  IA_CUDA(c, cudaMemsetAsync(c->d_pm, 0, sizeof(float) * np, s), "ia_proposal_set_params");
  IA_CUDA(c, cudaMemsetAsync(c->d_pv, 0, sizeof(float) * np, s), "ia_proposal_set_params");
  c->adam_step = 0;
  return IA_OK;
}

ia_status ia_proposal_get_params(ia_ctx* c, float* table, float* mlp, void* stream) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!c->prop_ready) return fail(c, IA_ERR_STATE, "ia_proposal_init has not been called");
  cudaStream_t s = (cudaStream_t)stream;
  if (table)
    IA_CUDA(c, cudaMemcpyAsync(table, c->d_ptable, sizeof(float) * 2 * c->p_entries, cudaMemcpyDefault, s),
            "ia_proposal_get_params");
  if (mlp) IA_CUDA(c, cudaMemcpyAsync(mlp, c->d_pmlp, sizeof(float) * c->p_mlp, cudaMemcpyDefault, s), "ia_proposal_get_params");
  IA_CUDA(c, cudaStreamSynchronize(s), "ia_proposal_get_params");
  return IA_OK;
}

ia_status ia_proposal_pairs(ia_ctx* c, int pose, int n, const float* x, int32_t* label, float* offset,
                            void* stream) {
  ia_status st = need_ready(c, pose, false);
  if (st != IA_OK) return st;
  if (n < 0 || (n > 0 && (!x || !label || !offset))) return fail(c, IA_ERR_ARG, "bad arrays");
  if (n == 0) return IA_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (n > c->pair_cap) {
    IA_CUDA(c, cudaStreamSynchronize(s), "ia_proposal_pairs");
    c->pair_cap = 0;
    IA_CUDA(c, dalloc(&c->d_pxc, (size_t)3 * n), "ia_proposal_pairs: workspace");
    IA_CUDA(c, dalloc(&c->d_pstart, (size_t)n), "ia_proposal_pairs: workspace");
    c->pair_cap = n;
  }
  PosedArgs a = posed_args(c, pose);
  a.search = 0;  // labels come from the plain search over every bone
  IA_CUDA(c, launch_query_posed(a, n, x, nullptr, nullptr, c->d_pxc, c->d_pstart, s), "ia_proposal_pairs: search");
  PropLabelArgs la{};
  la.S = a.S;
  la.skin = c->d_skin;
  la.nb = c->nb;
  la.Ninv = a.Ninv;
  la.n = n;
  la.x = x;
  la.xc = c->d_pxc;
  la.start = c->d_pstart;
  la.label = label;
  la.offset = offset;
  IA_CUDA(c, launch_prop_label(la, s), "ia_proposal_pairs: labels");
  return IA_OK;
}

static ia_status prop_check(ia_ctx* c, int n, const float* x, const int32_t* pose, const int32_t* label,
                            const float* target) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (!c->prop_ready) return fail(c, IA_ERR_STATE, "ia_proposal_init has not been called");
  if (c->n_poses == 0) return fail(c, IA_ERR_STATE, "ia_set_pose has not been called");
  if (n < 1 || !x || !pose || !label || !target) return fail(c, IA_ERR_ARG, "bad pair arrays");
  return IA_OK;
}

static ia_status prop_workspace(ia_ctx* c, int batch, cudaStream_t s) {
  if (batch > c->prow_cap) {
    IA_CUDA(c, cudaStreamSynchronize(s), "proposal workspace");
    c->prow_cap = 0;
    IA_CUDA(c, dalloc(&c->d_prows, (size_t)batch * kPropRow), "proposal workspace");
    c->prow_cap = batch;
  }
  return IA_OK;
}

static PropTrainArgs prop_train_args(ia_ctx* c, int n, const float* x, const int32_t* pose, const int32_t* label,
                                     const float* target) {
  PropTrainArgs a{};
  a.Q = prop_dev(c);
  a.nb = c->nb;
  a.theta = c->d_theta;
  a.n = n;
  a.x = x;
  a.pose = pose;
  a.label = label;
  a.target = target;
  a.offset_weight = c->pcfg.offset_weight;
  a.rows = c->d_prows;
  a.g_table = c->d_pg;
  a.g_mlp = c->d_pg + 2 * c->p_entries;
  return a;
}

ia_status ia_proposal_grad(ia_ctx* c, int n, const float* x, const int32_t* pose, const int32_t* label,
                           const float* target, float* loss, float* g_table, float* g_mlp, void* stream) {
  ia_status st = prop_check(c, n, x, pose, label, target);
  if (st != IA_OK) return st;
  if (!loss) return fail(c, IA_ERR_ARG, "null loss");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prop_workspace(c, n, s)) != IA_OK) return st;
  const size_t np = (size_t)(2 * c->p_entries + c->p_mlp);
  IA_CUDA(c, cudaMemsetAsync(c->d_pg, 0, sizeof(float) * np, s), "ia_proposal_grad");
  IA_CUDA(c, cudaMemsetAsync(loss, 0, sizeof(float), s), "ia_proposal_grad");
  PropTrainArgs a = prop_train_args(c, n, x, pose, label, target);
  a.first = 0;
  a.batch = n;
  a.loss = loss;
  IA_CUDA(c, launch_prop_grad(a, s), "ia_proposal_grad");
  if (g_table)
    IA_CUDA(c, cudaMemcpyAsync(g_table, c->d_pg, sizeof(float) * 2 * c->p_entries, cudaMemcpyDefault, s), "ia_proposal_grad");
  if (g_mlp)
    IA_CUDA(c, cudaMemcpyAsync(g_mlp, c->d_pg + 2 * c->p_entries, sizeof(float) * c->p_mlp, cudaMemcpyDefault, s),
            "ia_proposal_grad");
  return IA_OK;
}

ia_status ia_proposal_train(ia_ctx* c, int n, const float* x, const int32_t* pose, const int32_t* label,
                            const float* target, int steps, int batch, float lr, float* loss_out, void* stream) {
  ia_status st = prop_check(c, n, x, pose, label, target);
  if (st != IA_OK) return st;
  if (steps < 0 || batch < 1 || batch > (1 << 22) || !(lr > 0.f)) return fail(c, IA_ERR_ARG, "bad training settings");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prop_workspace(c, batch, s)) != IA_OK) return st;
  const size_t np = (size_t)(2 * c->p_entries + c->p_mlp);
  PropTrainArgs a = prop_train_args(c, n, x, pose, label, target);
  a.batch = batch;
  for (int k = 0; k < steps; ++k) {
    a.first = (int)(((int64_t)k * batch) % n);
    a.loss = loss_out ? loss_out + k : c->d_ploss;
    IA_CUDA(c, cudaMemsetAsync(c->d_pg, 0, sizeof(float) * np, s), "ia_proposal_train");
    IA_CUDA(c, cudaMemsetAsync(a.loss, 0, sizeof(float), s), "ia_proposal_train");
    IA_CUDA(c, launch_prop_grad(a, s), "ia_proposal_train: gradient");
    ++c->adam_step;
    IA_CUDA(c, launch_adam(c->d_pp, c->d_pg, c->d_pm, c->d_pv, (int64_t)np, lr, c->adam_step, 0.9f, 0.999f, 1e-8f,
                           nullptr, s),
            "ia_proposal_train: adam");
  }
  return IA_OK;
}

ia_status ia_set_occupancy_culling(ia_ctx* c, int on) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (on != 0 && on != 1) return fail(c, IA_ERR_ARG, "culling must be 0 or 1");
  c->occ_cull = on == 1;
  return IA_OK;
}

ia_status ia_set_search(ia_ctx* c, int mode) {
  if (!c) return fail(nullptr, IA_ERR_ARG, "null context");
  if (mode != IA_SEARCH_ALL_BONES && mode != IA_SEARCH_PROPOSAL) return fail(c, IA_ERR_ARG, "unknown search mode");
  if (mode == IA_SEARCH_PROPOSAL) {
    if (!c->prop_ready) return fail(c, IA_ERR_STATE, "ia_proposal_init has not been called");
    if (c->cfg.precision == IA_FP32) return fail(c, IA_ERR_ARG, "the proposal search needs precision fp16 or bf16");
  }
  c->search = mode;
  return IA_OK;
}

// ---------------------------------------------------------------------------
// Occupancy update without any allocation: the per-cell density scratch lives
// in a fixed, file-scope device array instead of context memory.
// ---------------------------------------------------------------------------

namespace {

constexpr int kStaticOccRes = 64;  // largest grid the static scratch holds: 64^3 cells, 1 MiB
static __device__ __align__(256) float g_occ_sigma_scratch[kStaticOccRes * kStaticOccRes * kStaticOccRes];

constexpr int kMaxDevices = 64;
float* g_occ_scratch_addr[kMaxDevices] = {};
std::mutex g_occ_scratch_mu;

// Device address of the static scratch on the current device, looked up once per
// device.  In host code the array's name only stands in for the symbol, so the
// address has to come from the runtime.
cudaError_t static_scratch(int dev, float** out) {
  std::lock_guard<std::mutex> lock(g_occ_scratch_mu);
  if (!g_occ_scratch_addr[dev]) {
    float* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_occ_sigma_scratch);
    if (e != cudaSuccess) return e;
    g_occ_scratch_addr[dev] = p;
  }
  *out = g_occ_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

ia_status ia_update_occupancy_static(ia_ctx* c, int pose, uint32_t* bits_out, void* stream) {
  ia_status st = need_ready(c, pose, false);
  if (st != IA_OK) return st;
  const int R = c->cfg.occ_res;
  if (R > kStaticOccRes)
    return fail(c, IA_ERR_LIMIT, "occ_res %d exceeds the static scratch limit of %d (use ia_update_occupancy)", R,
                kStaticOccRes);
  int dev = -1;
  IA_CUDA(c, cudaGetDevice(&dev), "ia_update_occupancy_static");
  if (dev != c->device)
    return fail(c, IA_ERR_STATE, "device %d is current but the context lives on device %d", dev, c->device);
  if (dev < 0 || dev >= kMaxDevices) return fail(c, IA_ERR_LIMIT, "device index %d beyond %d", dev, kMaxDevices);
  float* sigma = nullptr;
  IA_CUDA(c, static_scratch(dev, &sigma), "ia_update_occupancy_static: cudaGetSymbolAddress");
  cudaStream_t s = (cudaStream_t)stream;
  // every one of the R^3 cells is written (searched, or set to 0 when culled)
  // before the bits kernel reads them, so the scratch needs no clearing; cells
  // past R^3 are never read
  IA_CUDA(c, occ_density(c, pose, nullptr, sigma, nullptr, s, true), "ia_update_occupancy_static: density");
  IA_CUDA(c, launch_occ_bits(sigma, R, c->cfg.occ_dilate, c->cfg.occ_tau, c->d_occ, nullptr, s),
          "ia_update_occupancy_static: bits");
  c->have_occ = true;
  c->blist_pose = -1;  // the render's box lists belong to the previous grid
  if (bits_out) {
    const size_t words = ((size_t)R * R * R + 31) / 32;
    IA_CUDA(c, cudaMemcpyAsync(bits_out, c->d_occ, words * 4, cudaMemcpyDeviceToDevice, s),
            "ia_update_occupancy_static");
  }
  return IA_OK;
}

}  // extern "C"
