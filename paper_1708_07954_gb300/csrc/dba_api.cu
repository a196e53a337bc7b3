// Host side of the C ABI declared in include/dba.h: validation, the
// observation layout (sort by point, tiles of whole tracks, segmented-run
// tables), device memory, CUDA-graph replay of one ADMM iteration, metrics
// and state transfer.  Every step of the iteration itself runs in the kernels
// of dba_kernels.cu; the host only prepares static index tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dba.h"
#include "dba_internal.h"
#include "dba_guard.h"

using dba::DevCtl;
using dba::DevProblem;
using dba::Params;

namespace {
thread_local std::string g_create_error = "no error";

struct HostLayout {
  std::vector<long long> perm;  // internal position -> caller index
  std::vector<int> pt_perm;     // internal point -> caller point
  std::vector<int> obs_pt;      // internal point of each observation
  std::vector<int> obs_cam;     // camera of each observation
  std::vector<int> obs_cam_rank;  // camera | rank in the tile's camera order << 24
  std::vector<dba::TileInfo> tiles;
  std::vector<int> pseg_slot, cseg_slot;
  std::vector<int2> pseg, cseg;
  std::vector<int> cam_slot_off, cam_count, split_pt, split_slot_off{0}, pt_count;
  int n_cam_slots = 0, n_pt_slots = 0;
};

// Runs f(t, lo, hi) on T threads over contiguous chunks of [0, n).
template <typename F>
void parallel_chunks(long long n, int T, F f) {
  if (T <= 1) {
    f(0, 0LL, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T);
  for (int t = 0; t < T; ++t) th.emplace_back(f, t, n * t / T, n * (t + 1) / T);
  for (std::thread& x : th) x.join();
}

int host_threads(long long work) {
  if (work < (1LL << 16)) return 1;
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hw ? hw : 1u, 16u));
}

bool finite_all(const double* p, long long n) {
  const int T = host_threads(n);
  std::vector<char> ok(T, 1);
  parallel_chunks(n, T, [&](int t, long long lo, long long hi) {
    for (long long k = lo; k < hi; ++k)
      if (!std::isfinite(p[k])) {
        ok[t] = 0;
        return;
      }
  });
  for (char c : ok)
    if (!c) return false;
  return true;
}

// First observation whose point or camera index is out of range, or -1.
long long first_bad_index(const int32_t* pt_idx, const int32_t* cam_idx, long long n_obs, int n_pts, int n_cams) {
  const int T = host_threads(n_obs);
  std::vector<long long> bad(T, -1);
  parallel_chunks(n_obs, T, [&](int t, long long lo, long long hi) {
    for (long long o = lo; o < hi; ++o)
      if (pt_idx[o] < 0 || pt_idx[o] >= n_pts || cam_idx[o] < 0 || cam_idx[o] >= n_cams) {
        bad[t] = o;
        return;
      }
  });
  for (long long b : bad)
    if (b >= 0) return b;  // chunks are in order: the first hit is the smallest index
  return -1;
}
}  // namespace

struct dba_ctx {
  dba_config cfg;
  Params prm;
  std::string err = "no error";
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool fp32 = true;
  int fin_threads = 128;  // block size of finalize for the loaded problem
  // problem
  bool has_problem = false, has_gt = false;
  int n_cams = 0, n_pts = 0;
  long long n_obs = 0;
  std::vector<long long> perm;   // internal position -> caller index
  std::vector<int> pt_perm;      // internal point -> caller point
  std::vector<int> h_obs_pt, h_obs_cam;
  int64_t n_pseg = 0;
  int n_scenes = 0;
  bool warm = false;
  unsigned char* d_mlp_blob = nullptr;  // BF16 operands of the warm-start network
  float* d_mlp_params = nullptr;        // FP32 parameters (biases, normaliser)
  int* d_scene_of_obs = nullptr;   // [l] internal order
  double* d_scene_sums = nullptr;  // [n_scenes][5]
  std::vector<void*> allocs;
  DevProblem P{};
  dba::TileMaps tmaps{};  // tensor maps of P's observation arrays (tile kernel staging)
  int cur = 0, pending = 0;
  long long iters = 0;
  // graph of one iteration
  cudaGraphExec_t graph = nullptr;        // one iteration
  cudaGraphExec_t graph_until = nullptr;  // one iteration and the reference-pixel metrics pass
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  double rho_of(int c) const { return c < 3 ? prm.rho_x : (c < 6 ? prm.rho_a : prm.rho_y); }
  dba_status fail(dba_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  dba_status cuda_fail(cudaError_t e, const char* where) {
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return DBA_ECUDA;
  }
  void drop_graphs() {  // after any change of the captured kernel arguments
    if (graph) cudaGraphExecDestroy(graph);
    if (graph_until) cudaGraphExecDestroy(graph_until);
    graph = graph_until = nullptr;
  }
  void free_problem() {
    drop_graphs();
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    P = DevProblem{};
    has_problem = has_gt = false;
    n_scenes = 0;
    warm = false;
    d_mlp_blob = nullptr;
    d_mlp_params = nullptr;
    d_scene_of_obs = nullptr;
    d_scene_sums = nullptr;
    perm.clear();
    pt_perm.clear();
    h_obs_pt.clear();
    h_obs_cam.clear();
  }
  template <typename V>
  cudaError_t alloc(V** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(V));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    *out = static_cast<V*>(p);
    return cudaSuccess;
  }
  template <typename V>
  cudaError_t upload(const V** out, const std::vector<V>& h) {
    V* d = nullptr;
    cudaError_t e = alloc(&d, h.size());
    if (e != cudaSuccess) return e;
    if (!h.empty()) e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, stream);
    *out = d;
    return e;
  }
};

#define DBA_CUDA(call, where)                           \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ctx->cuda_fail(e_, where); \
  } while (0)

namespace {

// Observation layout.  Points are ordered by their smallest camera index (so a
// tile's tracks share cameras) and renumbered internally in that order, so
// every tile covers a contiguous range of internal point ids; each point's
// observations are sorted by camera.  Tiles hold whole tracks of at most
// tile_obs observations; a longer track is cut into tile-sized pieces reduced
// in the finalize kernel.  Within a tile, observations of one camera form runs
// in camera order; an observation's position in that order is packed above its
// camera index.
void build_layout(int n_cams, int n_pts, long long n_obs, const int32_t* pt_idx,
                  const int32_t* cam_idx, int NT, HostLayout& L) {
  const int T = host_threads(n_obs);
  // per-thread histograms of contiguous observation chunks: points (also giving each chunk
  // its own slots within every point, a stable counting sort) and cameras; first camera of
  // each point per chunk
  std::vector<std::vector<int>> hist(T), camc(T), first(T);
  parallel_chunks(n_obs, T, [&](int t, long long lo, long long hi) {
    hist[t].assign(n_pts, 0);
    camc[t].assign(n_cams, 0);
    first[t].assign(n_pts, n_cams);
    for (long long o = lo; o < hi; ++o) {
      const int i = pt_idx[o], j = cam_idx[o];
      hist[t][i] += 1;
      camc[t][j] += 1;
      if (j < first[t][i]) first[t][i] = j;
    }
  });
  std::vector<int> count(n_pts, 0), min_cam(n_pts, n_cams);
  parallel_chunks(n_pts, T, [&](int, long long lo, long long hi) {
    for (long long i = lo; i < hi; ++i)
      for (int t = 0; t < T; ++t) {
        count[i] += hist[t][i];
        min_cam[i] = std::min(min_cam[i], first[t][i]);
      }
  });
  first.clear();
  L.cam_count.assign(n_cams, 0);
  for (int t = 0; t < T; ++t)
    for (int j = 0; j < n_cams; ++j) L.cam_count[j] += camc[t][j];
  // internal point numbering: observed points by first camera (ties by index: a counting
  // sort over first cameras), then unobserved ones (first camera n_cams)
  std::vector<int> order(n_pts), inv(n_pts);
  {
    std::vector<int> fc(n_cams + 2, 0);
    for (int i = 0; i < n_pts; ++i) fc[min_cam[i] + 1] += 1;
    for (int j = 0; j <= n_cams; ++j) fc[j + 1] += fc[j];
    for (int i = 0; i < n_pts; ++i) order[fc[min_cam[i]]++] = i;
  }
  L.pt_perm = order;
  L.pt_count.resize(n_pts);
  for (int k = 0; k < n_pts; ++k) {
    L.pt_count[k] = count[order[k]];
    inv[order[k]] = k;
  }
  int n_obs_pts = 0;
  while (n_obs_pts < n_pts && L.pt_count[n_obs_pts] > 0) ++n_obs_pts;
  std::vector<long long> kpos(n_pts + 1, 0);  // first internal position of each internal point
  for (int k = 0; k < n_pts; ++k) kpos[k + 1] = kpos[k] + L.pt_count[k];

  // observations scattered straight into internal order (a stable counting sort by
  // point: chunk t's observations of a point follow those of chunks before it), with
  // their cameras alongside
  L.perm.resize(n_obs);
  L.obs_pt.resize(n_obs);
  L.obs_cam.resize(n_obs);
  L.obs_cam_rank.resize(n_obs);
  parallel_chunks(n_pts, T, [&](int, long long lo, long long hi) {
    for (long long i = lo; i < hi; ++i) {
      long long off = kpos[inv[i]];
      for (int t = 0; t < T; ++t) {
        const int c = hist[t][i];
        hist[t][i] = (int)off;  // first position of chunk t's observations of point i
        off += c;
      }
    }
  });
  parallel_chunks(n_obs, T, [&](int t, long long lo, long long hi) {
    std::vector<int>& h = hist[t];
    for (long long o = lo; o < hi; ++o) {
      const int q = h[pt_idx[o]]++;
      L.perm[q] = o;
      L.obs_cam[q] = cam_idx[o];
    }
  });
  // each point's observations by camera, ties in caller order (the scatter left them in
  // caller order, so a stable sort by camera)
  parallel_chunks(n_obs_pts, T, [&](int, long long lo, long long hi) {
    std::vector<std::pair<int, long long>> pr;
    for (long long k = lo; k < hi; ++k) {
      const long long s = kpos[k];
      const int c = L.pt_count[k];
      long long* bo = L.perm.data() + s;
      int* bc = L.obs_cam.data() + s;
      if (c <= 32) {
        for (int a = 1; a < c; ++a) {
          const int kc = bc[a];
          const long long ko = bo[a];
          int b = a - 1;
          for (; b >= 0 && bc[b] > kc; --b) {
            bc[b + 1] = bc[b];
            bo[b + 1] = bo[b];
          }
          bc[b + 1] = kc;
          bo[b + 1] = ko;
        }
      } else {
        pr.resize(c);
        for (int q = 0; q < c; ++q) pr[q] = {bc[q], bo[q]};
        std::sort(pr.begin(), pr.end());
        for (int q = 0; q < c; ++q) {
          bc[q] = pr[q].first;
          bo[q] = pr[q].second;
        }
      }
      for (int q = 0; q < c; ++q) L.obs_pt[s + q] = (int)k;
    }
  });

  // tiles of whole tracks; a track longer than a tile is split over tiles of its own
  long long pos = 0;
  int fill_tile = 0;           // observations in the open tile
  long long tile_start = 0;    // first observation of the open tile
  int tile_first_run = 0;      // first point run of the open tile
  int tile_first_pt = 0;       // first internal point of the open tile
  auto close_tile = [&]() {
    dba::TileInfo ti{};
    ti.o0 = (int)tile_start;
    ti.n = (int)(pos - tile_start);
    ti.r0 = tile_first_run;
    ti.nr = (int)L.pseg.size() - tile_first_run;
    ti.pt_lo = tile_first_pt;
    L.tiles.push_back(ti);
    tile_start = pos;
    tile_first_run = (int)L.pseg.size();
    fill_tile = 0;
  };
  for (int k = 0; k < n_obs_pts; ++k) {
    const int c = L.pt_count[k];
    if (c <= NT) {
      if (fill_tile + c > NT) close_tile();
      if (fill_tile == 0) tile_first_pt = k;
      L.pseg.push_back(make_int2(fill_tile, c));
      L.pseg_slot.push_back(-1);
      fill_tile += c;
      pos += c;
    } else {
      if (fill_tile > 0) close_tile();
      L.split_pt.push_back(k);
      int rem = c;
      while (rem > 0) {
        const int take = std::min(rem, NT);
        tile_first_pt = k;
        L.pseg.push_back(make_int2(0, take));
        L.pseg_slot.push_back(L.n_pt_slots++);
        fill_tile = take;
        pos += take;
        rem -= take;
        if (rem > 0) close_tile();
      }
      L.split_slot_off.push_back(L.n_pt_slots);
    }
  }
  if (fill_tile > 0) close_tile();

  // camera runs per tile, in camera order: each thread handles a contiguous range of
  // tiles into its own run lists, concatenated in tile order afterwards
  const long long n_tiles = (long long)L.tiles.size();
  const int Tt = std::max(1, std::min(T, (int)(n_tiles / 64)));
  std::vector<std::vector<int2>> t_cseg(Tt);
  std::vector<std::vector<int>> t_cam(Tt);
  parallel_chunks(n_tiles, Tt, [&](int t, long long lo, long long hi) {
    std::vector<int> idx;
    std::vector<unsigned long long> key;
    for (long long q0 = lo; q0 < hi; ++q0) {
      dba::TileInfo& ti = L.tiles[q0];
      // the tile's observations by camera, ties in tile order: sort (camera, position) keys
      key.resize(ti.n);
      for (int q = 0; q < ti.n; ++q)
        key[q] = ((unsigned long long)(unsigned)L.obs_cam[ti.o0 + q] << 32) | (unsigned)q;
      std::sort(key.begin(), key.end());
      idx.resize(ti.n);
      for (int q = 0; q < ti.n; ++q) idx[q] = ti.o0 + (int)(key[q] & 0xffffffffu);
      for (int r = 0; r < (int)idx.size(); ++r) L.obs_cam_rank[idx[r]] = L.obs_cam[idx[r]] | (r << 24);
      ti.c0 = (int)t_cseg[t].size();  // local; shifted below
      int r = 0;
      while (r < (int)idx.size()) {
        int e = r;
        while (e < (int)idx.size() && L.obs_cam[idx[e]] == L.obs_cam[idx[r]]) ++e;
        t_cseg[t].push_back(make_int2(r, e - r));
        t_cam[t].push_back(L.obs_cam[idx[r]]);
        r = e;
      }
      ti.nc = (int)t_cseg[t].size() - ti.c0;
    }
  });
  std::vector<int> run_cam;
  {
    long long base = 0;
    for (int t = 0; t < Tt; ++t) {
      const long long lo = n_tiles * t / Tt, hi = n_tiles * (t + 1) / Tt;
      for (long long q0 = lo; q0 < hi; ++q0) L.tiles[q0].c0 += (int)base;
      L.cseg.insert(L.cseg.end(), t_cseg[t].begin(), t_cseg[t].end());
      run_cam.insert(run_cam.end(), t_cam[t].begin(), t_cam[t].end());
      base += (long long)t_cseg[t].size();
    }
  }
  // camera partial slots grouped by camera
  L.cam_slot_off.assign(n_cams + 1, 0);
  for (int cam : run_cam) L.cam_slot_off[cam + 1] += 1;
  for (int j = 0; j < n_cams; ++j) L.cam_slot_off[j + 1] += L.cam_slot_off[j];
  std::vector<int> cfill(L.cam_slot_off.begin(), L.cam_slot_off.end() - 1);
  L.cseg_slot.resize(run_cam.size());
  for (size_t r = 0; r < run_cam.size(); ++r) L.cseg_slot[r] = cfill[run_cam[r]]++;
  L.n_cam_slots = L.cam_slot_off[n_cams];
}

}  // namespace

extern "C" {

void dba_config_default(dba_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->focal = 500.0;
  cfg->cx = 320.0;
  cfg->cy = 240.0;
  cfg->loss = DBA_LOSS_HUBER;
  cfg->loss_param = 2.0;
  cfg->rho_x = 1.0;
  cfg->rho_y = 1.0;
  cfg->inner_steps = 5;
  cfg->lm_lambda0 = 1e-3;
  cfg->lm_lambda_min = 1e-12;
  cfg->eps_depth = 1e-6;
  cfg->lm_model_tol = 16.0;
  cfg->precision = DBA_PREC_F32_LOCAL;
  cfg->tile_obs = 0;
  cfg->use_graph = 1;
  cfg->cuda_stream = nullptr;
  cfg->local_solver = DBA_SOLVER_GN;
  cfg->finalize_threads = 0;
}

dba_status dba_create(const dba_config* cfg, dba_ctx** out) {
  return dba::guarded(&g_create_error, [&]() -> dba_status {
    if (!cfg || !out) {
      g_create_error = "dba_create: null argument";
      return DBA_EINVAL;
    }
    *out = nullptr;
    const bool ok = std::isfinite(cfg->focal) && cfg->focal > 0 && std::isfinite(cfg->cx) &&
                    std::isfinite(cfg->cy) && cfg->loss >= 0 && cfg->loss <= 2 &&
                    (cfg->loss == DBA_LOSS_L2 || (std::isfinite(cfg->loss_param) && cfg->loss_param > 0)) &&
                    std::isfinite(cfg->rho_x) && cfg->rho_x > 0 && std::isfinite(cfg->rho_y) &&
                    cfg->rho_y > 0 && std::isfinite(cfg->rho_angle) && cfg->inner_steps >= 0 && cfg->inner_steps <= 1000 &&
                    std::isfinite(cfg->lm_lambda0) && cfg->lm_lambda0 > 0 &&
                    std::isfinite(cfg->lm_lambda_min) && cfg->lm_lambda_min >= 0 &&
                    std::isfinite(cfg->eps_depth) && std::isfinite(cfg->lm_model_tol) &&
                    cfg->lm_model_tol >= 0 && (cfg->precision == 0 || cfg->precision == 1) &&
                    (cfg->tile_obs == 0 || cfg->tile_obs == -1 || cfg->tile_obs == 64 ||
                     cfg->tile_obs == 128 || cfg->tile_obs == 256) &&
                    (cfg->local_solver == DBA_SOLVER_GN || cfg->local_solver == DBA_SOLVER_LBFGS) &&
                    (cfg->finalize_threads == 0 || cfg->finalize_threads == 32 || cfg->finalize_threads == 64 ||
                     cfg->finalize_threads == 128 || cfg->finalize_threads == 256);
    if (!ok) {
      g_create_error =
          "dba_create: invalid configuration (check focal, loss, rho, steps, precision, tile_obs, local_solver, "
          "finalize_threads)";
      return DBA_EINVAL;
    }
    cudaError_t e = cudaFree(nullptr);  // initialise the runtime on the current device
    if (e == cudaSuccess) e = dba::prepare_tile_kernels();
    if (e != cudaSuccess) {
      g_create_error = std::string("dba_create: CUDA unavailable: ") + cudaGetErrorString(e);
      return DBA_ECUDA;
    }
    dba_ctx* ctx = new (std::nothrow) dba_ctx();
    if (!ctx) {
      g_create_error = "dba_create: out of host memory";
      return DBA_ENOMEM;
    }
    ctx->cfg = *cfg;
    ctx->fp32 = cfg->precision == DBA_PREC_F32_LOCAL;
    ctx->prm = Params{cfg->focal, cfg->cx, cfg->cy, cfg->loss, cfg->loss_param, cfg->rho_x, cfg->rho_y,
                      cfg->rho_angle > 0 ? cfg->rho_angle : cfg->rho_y,
                      cfg->inner_steps, cfg->lm_lambda0, cfg->lm_lambda_min, cfg->eps_depth,
                      cfg->lm_model_tol, cfg->local_solver};
    if (cfg->cuda_stream) {
      ctx->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        g_create_error = std::string("dba_create: ") + cudaGetErrorString(e);
        delete ctx;
        return DBA_ECUDA;
      }
      ctx->own_stream = true;
    }
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
      g_create_error = "dba_create: cudaEventCreate failed";
      if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
      delete ctx;
      return DBA_ECUDA;
    }
    *out = ctx;
    return DBA_OK;
  });
}

void dba_destroy(dba_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  ctx->free_problem();
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* dba_last_error(const dba_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

namespace {

template <typename T>
void to_T(const std::vector<double>& src, std::vector<T>& dst) {
  dst.resize(src.size());
  for (size_t k = 0; k < src.size(); ++k) dst[k] = (T)src[k];
}

// hdel / hdual empty: copies at the consensus (zero offsets) / zero duals, set on the device.
template <typename T>
dba_status upload_state_T(dba_ctx* ctx, const double* cams, const double* pts,
                          const std::vector<double>& hdel, const std::vector<double>& hdual, bool exact) {
  DevProblem& P = ctx->P;
  const int m = ctx->n_cams, n = ctx->n_pts;
  const size_t l = (size_t)ctx->n_obs, lp = (size_t)P.pitch;  // host rows dense, device rows pitched
  std::vector<T> tdel, tX, tY;
  to_T(hdel, tdel);
  to_T(std::vector<double>(pts, pts + 3 * (size_t)n), tX);
  to_T(std::vector<double>(cams, cams + 6 * (size_t)m), tY);
  cudaStream_t st = ctx->stream;
  if (tdel.empty())
    DBA_CUDA(cudaMemsetAsync(P.delta, 0, 9 * lp * sizeof(T), st), "clear copies");
  else
    DBA_CUDA(cudaMemcpy2DAsync(P.delta, lp * sizeof(T), tdel.data(), l * sizeof(T), l * sizeof(T), 9,
                               cudaMemcpyHostToDevice, st),
             "upload copies");
  if (hdual.empty())
    DBA_CUDA(cudaMemsetAsync(P.adual, 0, 9 * lp * sizeof(double), st), "clear duals");
  else
    DBA_CUDA(cudaMemcpy2DAsync(P.adual, lp * sizeof(double), hdual.data(), l * sizeof(double), l * sizeof(double), 9,
                               cudaMemcpyHostToDevice, st),
             "upload duals");
  for (int b = 0; b < 2; ++b) {
    DBA_CUDA(cudaMemcpyAsync(P.X[b], pts, 3 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st), "upload points");
    DBA_CUDA(cudaMemcpyAsync(P.Y[b], cams, 6 * (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st), "upload cameras");
  }
  DBA_CUDA(cudaMemcpyAsync(P.Xm, tX.data(), tX.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload points");
  DBA_CUDA(cudaMemcpyAsync(P.Ym, tY.data(), tY.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload cameras");
  DBA_CUDA(cudaMemsetAsync(P.DX, 0, 3 * (size_t)n * sizeof(T), st), "clear");
  DBA_CUDA(cudaMemsetAsync(P.DY, 0, 6 * (size_t)m * sizeof(T), st), "clear");
  DevCtl c0{};
  c0.exact = exact ? 1 : 0;
  DBA_CUDA(cudaMemcpyAsync(P.ctl, &c0, sizeof c0, cudaMemcpyHostToDevice, st), "clear");
  DBA_CUDA(cudaStreamSynchronize(st), "upload state");
  ctx->cur = 0;
  ctx->pending = 0;
  ctx->iters = 0;
  return DBA_OK;
}

// Copies given as absolute values are stored as offsets from the consensus;
// duals (r, s) are stored scaled by 1/rho.  NULL copies = consensus, NULL duals = 0.
dba_status upload_state(dba_ctx* ctx, const double* cams, const double* pts_caller, const double* copies,
                        const double* duals) {
  const long long l = ctx->n_obs;
  std::vector<double> pts_int(3 * (size_t)ctx->n_pts);
  for (int k = 0; k < ctx->n_pts; ++k)
    for (int c = 0; c < 3; ++c) pts_int[3 * (size_t)k + c] = pts_caller[3 * (size_t)ctx->pt_perm[k] + c];
  const double* pts = pts_int.data();
  std::vector<double> hdel, hdual;
  if (copies) hdel.assign(9 * (size_t)l, 0.0);
  if (duals) hdual.assign(9 * (size_t)l, 0.0);
  if (copies || duals) {
    for (long long o = 0; o < l; ++o) {
      const long long src = ctx->perm[o];
      const size_t i = ctx->h_obs_pt[o], j = ctx->h_obs_cam[o];
      for (int c = 0; c < 9; ++c) {
        if (copies) {
          const double cons = c < 3 ? pts[3 * i + c] : cams[6 * j + c - 3];
          hdel[c * (size_t)l + o] = copies[9 * src + c] - cons;
        }
        if (duals) hdual[c * (size_t)l + o] = duals[9 * src + c] / ctx->rho_of(c);
      }
    }
  }
  // with caller-supplied duals the per-point/camera dual sums need not vanish
  const bool exact = duals != nullptr;
  return ctx->fp32 ? upload_state_T<float>(ctx, cams, pts, hdel, hdual, exact)
                   : upload_state_T<double>(ctx, cams, pts, hdel, hdual, exact);
}

// launch = false reads the sums of a metrics pass already queued on the stream.
dba_status read_metrics(dba_ctx* ctx, dba_stats* st, double seconds, bool launch = true) {
  if (launch)
    DBA_CUDA(dba::launch_metrics(ctx->P, ctx->prm, ctx->fp32, ctx->cur, ctx->pending, ctx->stream),
             "metrics launch");
  double h[8];
  DBA_CUDA(cudaMemcpyAsync(h, ctx->P.metric_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "metrics copy");
  DBA_CUDA(cudaStreamSynchronize(ctx->stream), "metrics");
  const double valid = h[3];
  st->iters_done = ctx->iters;
  st->rmse_obs = valid > 0 ? std::sqrt(h[0] / valid) : 0.0;
  st->objective = h[1];
  st->rmse_gt = (h[7] > 0 && ctx->has_gt) ? std::sqrt(h[2] / h[7]) : 0.0;
  st->n_invalid = (long long)h[4];
  st->primal_res = std::sqrt(h[5]);
  st->dual_res = std::sqrt(h[6]);
  st->seconds = seconds;
  return DBA_OK;
}

dba_status launch_iteration(dba_ctx* ctx) {
  if (ctx->warm)
    DBA_CUDA(dba::launch_mlp_warmstart(ctx->P, ctx->prm, ctx->fp32, ctx->d_mlp_blob, ctx->d_mlp_params, ctx->stream),
             "warm start launch");
  DBA_CUDA(dba::launch_tile_iterate(ctx->P, ctx->tmaps, ctx->prm, ctx->fp32, ctx->stream), "tile_iterate launch");
  DBA_CUDA(dba::launch_finalize(ctx->P, ctx->fp32, ctx->stream), "finalize launch");
  return DBA_OK;
}

// with_metrics: the graph also runs the reference-pixel metrics pass after the iteration
// (its kernel arguments hold pending = 1, the state after any iteration).
dba_status ensure_graph(dba_ctx* ctx, bool with_metrics = false) {
  cudaGraphExec_t& exec = with_metrics ? ctx->graph_until : ctx->graph;
  if (exec) return DBA_OK;
  cudaGraph_t g = nullptr;
  DBA_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
  cudaError_t e0 = ctx->warm ? dba::launch_mlp_warmstart(ctx->P, ctx->prm, ctx->fp32, ctx->d_mlp_blob,
                                                          ctx->d_mlp_params, ctx->stream)
                             : cudaSuccess;
  cudaError_t e1 = dba::launch_tile_iterate(ctx->P, ctx->tmaps, ctx->prm, ctx->fp32, ctx->stream);
  cudaError_t e2 = dba::launch_finalize(ctx->P, ctx->fp32, ctx->stream);
  cudaError_t e4 = with_metrics ? dba::launch_metrics(ctx->P, ctx->prm, ctx->fp32, ctx->cur ^ 1, 1, ctx->stream, true)
                                : cudaSuccess;
  cudaError_t e3 = cudaStreamEndCapture(ctx->stream, &g);
  if (e0 != cudaSuccess) return ctx->cuda_fail(e0, "graph capture (warm start)");
  if (e1 != cudaSuccess) return ctx->cuda_fail(e1, "graph capture (tile_iterate)");
  if (e2 != cudaSuccess) return ctx->cuda_fail(e2, "graph capture (finalize)");
  if (e4 != cudaSuccess) return ctx->cuda_fail(e4, "graph capture (metrics)");
  if (e3 != cudaSuccess) return ctx->cuda_fail(e3, "graph capture");
  cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    exec = nullptr;
    return ctx->cuda_fail(e, "graph instantiate");
  }
  return DBA_OK;
}

dba_status run_iterations(dba_ctx* ctx, int n) {
  if (ctx->cfg.use_graph) {
    dba_status s = ensure_graph(ctx);
    if (s != DBA_OK) return s;
    for (int it = 0; it < n; ++it) DBA_CUDA(cudaGraphLaunch(ctx->graph, ctx->stream), "graph launch");
  } else {
    for (int it = 0; it < n; ++it) {
      dba_status s = launch_iteration(ctx);
      if (s != DBA_OK) return s;
    }
  }
  if (n > 0) {
    ctx->cur ^= (n & 1);
    ctx->pending = 1;
    ctx->iters += n;
  }
  return DBA_OK;
}

dba_status check_device_flags(dba_ctx* ctx) {
  DevCtl h{};
  DBA_CUDA(cudaMemcpyAsync(&h, ctx->P.ctl, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "read control");
  DBA_CUDA(cudaStreamSynchronize(ctx->stream), "iterate");
  if (h.err & 1) return ctx->fail(DBA_ENUMERIC, "a local solve produced a non-finite value");
  if (h.err & 2) return ctx->fail(DBA_ETIMEOUT, "a tensor-core wait of the warm-start network timed out");
  if (h.err & 4) return ctx->fail(DBA_ETIMEOUT, "a wait for the tile kernel's tensor copies timed out");
  if (h.cur != ctx->cur) return ctx->fail(DBA_ECUDA, "device control word out of step with the host");
  return DBA_OK;
}

}  // namespace

namespace {

// Builds the layout for tile size NT, uploads it and the initial state (copies at the
// initial estimate, zero duals).  Inputs are already validated.
dba_status load_problem(dba_ctx* ctx, int NT, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                        const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                        const double* cams0, const double* pts0) {
  HostLayout L;
  build_layout(n_cams, n_pts, n_obs, pt_idx, cam_idx, NT, L);
  ctx->n_cams = n_cams;
  ctx->n_pts = n_pts;
  ctx->n_obs = n_obs;
  ctx->perm = std::move(L.perm);
  ctx->pt_perm = L.pt_perm;
  ctx->h_obs_pt = L.obs_pt;
  ctx->h_obs_cam = L.obs_cam;
  ctx->n_pseg = (int64_t)L.pseg.size();

  DevProblem& P = ctx->P;
  P.n_cams = n_cams;
  P.n_pts = n_pts;
  P.n_obs = n_obs;
  P.n_tiles = (int)L.tiles.size();
  P.tile_obs = NT;
  P.fin_threads = ctx->fin_threads;
  P.n_cam_slots = L.n_cam_slots;
  P.n_pt_slots = L.n_pt_slots;
  P.n_split_pts = (int)L.split_pt.size();
  DBA_CUDA(ctx->upload(&P.obs_pt, L.obs_pt), "upload");
  DBA_CUDA(ctx->upload(&P.obs_cam_rank, L.obs_cam_rank), "upload");
  DBA_CUDA(ctx->upload(&P.tiles, L.tiles), "upload");
  DBA_CUDA(ctx->upload(&P.pseg, L.pseg), "upload");
  DBA_CUDA(ctx->upload(&P.pseg_slot, L.pseg_slot), "upload");
  DBA_CUDA(ctx->upload(&P.cseg, L.cseg), "upload");
  DBA_CUDA(ctx->upload(&P.cseg_slot, L.cseg_slot), "upload");
  DBA_CUDA(ctx->upload(&P.cam_slot_off, L.cam_slot_off), "upload");
  DBA_CUDA(ctx->upload(&P.cam_count, L.cam_count), "upload");
  DBA_CUDA(ctx->upload(&P.split_pt, L.split_pt), "upload");
  DBA_CUDA(ctx->upload(&P.split_slot_off, L.split_slot_off), "upload");
  DBA_CUDA(ctx->upload(&P.pt_count, L.pt_count), "upload");
  // observations in internal order
  const int T = host_threads(n_obs);
  if (ctx->fp32) {
    std::vector<float2> hz(n_obs);
    parallel_chunks(n_obs, T, [&](int, long long lo, long long hi) {
      for (long long o = lo; o < hi; ++o)
        hz[o] = make_float2((float)z[2 * ctx->perm[o]], (float)z[2 * ctx->perm[o] + 1]);
    });
    const float2* dz = nullptr;
    DBA_CUDA(ctx->upload(&dz, hz), "upload observations");
    P.z = dz;
  } else {
    std::vector<double2> hz(n_obs);
    parallel_chunks(n_obs, T, [&](int, long long lo, long long hi) {
      for (long long o = lo; o < hi; ++o) hz[o] = make_double2(z[2 * ctx->perm[o]], z[2 * ctx->perm[o] + 1]);
    });
    const double2* dz = nullptr;
    DBA_CUDA(ctx->upload(&dz, hz), "upload observations");
    P.z = dz;
  }
  const size_t esz = ctx->fp32 ? sizeof(float) : sizeof(double);
  char* p = nullptr;
  P.pitch = dba::obs_pitch(n_obs);
  DBA_CUDA(ctx->alloc(&p, 9 * (size_t)P.pitch * esz), "alloc copies");
  P.delta = p;
  DBA_CUDA(ctx->alloc(&P.adual, 9 * (size_t)P.pitch), "alloc duals");
  for (int b = 0; b < 2; ++b) {
    DBA_CUDA(ctx->alloc(&P.X[b], 3 * (size_t)n_pts), "alloc points");
    DBA_CUDA(ctx->alloc(&P.Y[b], 6 * (size_t)n_cams), "alloc cameras");
  }
  DBA_CUDA(ctx->alloc(&p, 3 * (size_t)n_pts * esz), "alloc");
  P.Xm = p;
  DBA_CUDA(ctx->alloc(&p, 3 * (size_t)n_pts * esz), "alloc");
  P.DX = p;
  DBA_CUDA(ctx->alloc(&p, 6 * (size_t)n_cams * esz), "alloc");
  P.Ym = p;
  DBA_CUDA(ctx->alloc(&p, 6 * (size_t)n_cams * esz), "alloc");
  P.DY = p;
  DBA_CUDA(ctx->alloc(&P.pt_part, 3 * (size_t)std::max(1, P.n_pt_slots)), "alloc partials");
  DBA_CUDA(ctx->alloc(&P.cam_part, 6 * (size_t)std::max(1, P.n_cam_slots)), "alloc partials");
  DBA_CUDA(ctx->alloc(&P.metric_part, 8 * (size_t)dba::kMetricBlocks), "alloc metrics");
  DBA_CUDA(ctx->alloc(&P.metric_out, 8), "alloc metrics");
  DBA_CUDA(ctx->alloc(&p, 12 * (size_t)n_cams * esz), "alloc camera poses");
  P.cam_pose = p;
  DBA_CUDA(ctx->alloc(&P.ctl, 1), "alloc control");
  DBA_CUDA(dba::encode_tile_maps(P, ctx->fp32, &ctx->tmaps), "tensor maps");
  ctx->has_problem = true;
  dba_status s = upload_state(ctx, cams0, pts0, nullptr, nullptr);
  if (s != DBA_OK) {
    ctx->free_problem();
    return s;
  }
  return DBA_OK;
}

// Autotuner of the two launch sizes of an iteration: the tile size (observations per tile
// and threads per block of tile_iterate, 64 / 128 / 256) and the block size of finalize's
// segmented reduction (32 / 64 / 128 / 256, unless the configuration fixes it).  For each
// tile size it loads the problem, and for each finalize size it times a few iterations; it
// keeps the fastest pair, and the caller reloads the problem with it (so the state is the
// initial one).  Results are cached per process by precision, problem size (power of two),
// mean track length and the fixed finalize size.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tune_cache;

dba_status autotune_tile(dba_ctx* ctx, int32_t n_cams, int32_t n_pts, int64_t n_obs, const int32_t* pt_idx,
                         const int32_t* cam_idx, const double* z, const double* cams0, const double* pts0,
                         int* best, int* best_fin) {
  int used = 0;
  {
    std::vector<char> seen(n_pts, 0);
    for (int64_t o = 0; o < n_obs; ++o) seen[pt_idx[o]] = 1;
    for (char c : seen) used += c;
  }
  int lg = 0;
  while ((1ll << (lg + 1)) <= n_obs) ++lg;
  const int mean_track = (int)std::lround((double)n_obs / std::max(1, used));
  const int fixed_fin = ctx->cfg.finalize_threads;
  const auto key = std::make_tuple(ctx->fp32 ? 1 : 0, lg, std::min(mean_track, 64), fixed_fin);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *best = it->second.first;
      *best_fin = it->second.second;
      return DBA_OK;
    }
  }
  const int candidates[3] = {64, 128, 256};
  const int fin_all[4] = {32, 64, 128, 256};
  const int n_fin = fixed_fin > 0 ? 1 : 4;
  const int* fin_candidates = fixed_fin > 0 ? &fixed_fin : fin_all;
  float best_ms = 0.f;
  *best = ctx->fp32 ? 256 : 128;
  *best_fin = fixed_fin > 0 ? fixed_fin : 128;
  const int reps = 3;
  for (int nt : candidates) {
    dba_status s = load_problem(ctx, nt, n_cams, n_pts, n_obs, pt_idx, cam_idx, z, cams0, pts0);
    if (s != DBA_OK) return s;
    for (int f = 0; f < n_fin; ++f) {
      ctx->P.fin_threads = fin_candidates[f];  // launched directly below, not from a graph
      s = launch_iteration(ctx);               // warm-up
      if (s != DBA_OK) return s;
      DBA_CUDA(cudaEventRecord(ctx->ev0, ctx->stream), "autotune");
      for (int r = 0; r < reps; ++r) {
        s = launch_iteration(ctx);
        if (s != DBA_OK) return s;
      }
      DBA_CUDA(cudaEventRecord(ctx->ev1, ctx->stream), "autotune");
      DBA_CUDA(cudaEventSynchronize(ctx->ev1), "autotune");
      float ms = 0.f;
      DBA_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "autotune");
      if (best_ms == 0.f || ms < best_ms) {
        best_ms = ms;
        *best = nt;
        *best_fin = fin_candidates[f];
      }
    }
    ctx->free_problem();
  }
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = {*best, *best_fin};
  return DBA_OK;
}

}  // namespace

extern "C" {

dba_status dba_set_observations(dba_ctx* ctx, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                                const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                                const double* cams0, const double* pts0) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0)
      return ctx->fail(DBA_EINVAL, "dba_set_observations: n_cams, n_pts and n_obs must be positive");
    if (n_obs > (int64_t)0x7fffffff)
      return ctx->fail(DBA_EINVAL, "dba_set_observations: at most 2^31-1 observations");
    if (n_cams > dba::kCamMask)
      return ctx->fail(DBA_EINVAL, "dba_set_observations: at most 16,777,215 cameras");
    if (!pt_idx || !cam_idx || !z || !cams0 || !pts0)
      return ctx->fail(DBA_EINVAL, "dba_set_observations: null array");
    const long long bad = first_bad_index(pt_idx, cam_idx, n_obs, n_pts, n_cams);
    if (bad >= 0)
      return ctx->fail(DBA_EINVAL, "dba_set_observations: observation " + std::to_string(bad) +
                                       " has an index out of range");
    if (!finite_all(z, 2 * n_obs) || !finite_all(cams0, 6 * (long long)n_cams) ||
        !finite_all(pts0, 3 * (long long)n_pts))
      return ctx->fail(DBA_EINVAL, "dba_set_observations: non-finite input value");
    cudaStreamSynchronize(ctx->stream);
    ctx->free_problem();
    int NT = ctx->cfg.tile_obs > 0 ? ctx->cfg.tile_obs : (ctx->fp32 ? 256 : 128);
    ctx->fin_threads = ctx->cfg.finalize_threads > 0 ? ctx->cfg.finalize_threads : 128;
    if (ctx->cfg.tile_obs < 0) {
      int NF = ctx->fin_threads;
      dba_status s = autotune_tile(ctx, n_cams, n_pts, n_obs, pt_idx, cam_idx, z, cams0, pts0, &NT, &NF);
      if (s != DBA_OK) return s;
      ctx->fin_threads = NF;
    }
    return load_problem(ctx, NT, n_cams, n_pts, n_obs, pt_idx, cam_idx, z, cams0, pts0);
  });
}

dba_status dba_set_ground_truth(dba_ctx* ctx, const double* cams_gt, const double* pts_gt,
                                const uint8_t* inlier) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_set_ground_truth before dba_set_observations");
    if (!cams_gt || !pts_gt) return ctx->fail(DBA_EINVAL, "dba_set_ground_truth: null array");
    if (!finite_all(cams_gt, 6 * (long long)ctx->n_cams) || !finite_all(pts_gt, 3 * (long long)ctx->n_pts))
      return ctx->fail(DBA_EINVAL, "dba_set_ground_truth: non-finite value");
    double *dc = nullptr, *dp = nullptr;
    cudaStream_t st = ctx->stream;
    DBA_CUDA(cudaMallocAsync(&dc, 6 * (size_t)ctx->n_cams * sizeof(double), st), "alloc");
    DBA_CUDA(cudaMallocAsync(&dp, 3 * (size_t)ctx->n_pts * sizeof(double), st), "alloc");
    DBA_CUDA(cudaMemcpyAsync(dc, cams_gt, 6 * (size_t)ctx->n_cams * sizeof(double), cudaMemcpyHostToDevice, st), "upload");
    std::vector<double> pts_int(3 * (size_t)ctx->n_pts);
    for (int k = 0; k < ctx->n_pts; ++k)
      for (int c = 0; c < 3; ++c) pts_int[3 * (size_t)k + c] = pts_gt[3 * (size_t)ctx->pt_perm[k] + c];
    DBA_CUDA(cudaMemcpyAsync(dp, pts_int.data(), pts_int.size() * sizeof(double), cudaMemcpyHostToDevice, st),
             "upload");
    void* zt = const_cast<void*>(ctx->P.zt);
    if (!zt) {
      char* p = nullptr;
      DBA_CUDA(ctx->alloc(&p, (size_t)ctx->n_obs * (ctx->fp32 ? sizeof(float2) : sizeof(double2))), "alloc");
      zt = p;
    }
    DBA_CUDA(dba::launch_project_truth(ctx->P, ctx->prm, ctx->fp32, dc, dp, zt, st), "project truth");
    if (inlier) {
      std::vector<unsigned char> h(ctx->n_obs);
      for (long long o = 0; o < ctx->n_obs; ++o) h[o] = inlier[ctx->perm[o]] ? 1 : 0;
      if (!ctx->P.inlier) {
        DBA_CUDA(ctx->upload(&ctx->P.inlier, h), "upload inlier mask");
      } else {
        DBA_CUDA(cudaMemcpyAsync(const_cast<unsigned char*>(ctx->P.inlier), h.data(), h.size(),
                                 cudaMemcpyHostToDevice, st), "upload inlier mask");
      }
      DBA_CUDA(cudaStreamSynchronize(st), "upload inlier mask");
    } else {
      ctx->P.inlier = nullptr;
    }
    DBA_CUDA(cudaFreeAsync(dc, st), "free");
    DBA_CUDA(cudaFreeAsync(dp, st), "free");
    DBA_CUDA(cudaStreamSynchronize(st), "ground truth");
    ctx->P.zt = zt;
    ctx->has_gt = true;
    ctx->drop_graphs();  // kernel arguments changed
    return DBA_OK;
  });
}

dba_status dba_iterate(dba_ctx* ctx, int n_iters, dba_stats* stats) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_iterate before dba_set_observations");
    if (n_iters < 0) return ctx->fail(DBA_EINVAL, "dba_iterate: n_iters < 0");
    DBA_CUDA(cudaEventRecord(ctx->ev0, ctx->stream), "event");
    dba_status s = run_iterations(ctx, n_iters);
    if (s != DBA_OK) return s;
    DBA_CUDA(cudaEventRecord(ctx->ev1, ctx->stream), "event");
    s = check_device_flags(ctx);
    if (s != DBA_OK) return s;
    float ms = 0.f;
    DBA_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "event");
    if (stats) return read_metrics(ctx, stats, ms * 1e-3);
    return DBA_OK;
  });
}

dba_status dba_iterate_until(dba_ctx* ctx, int max_iters, double target_rmse_gt, dba_stats* stats) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_iterate_until before dba_set_observations");
    if (!ctx->has_gt) return ctx->fail(DBA_ESTATE, "dba_iterate_until needs dba_set_ground_truth");
    if (max_iters < 0) return ctx->fail(DBA_EINVAL, "dba_iterate_until: max_iters < 0");
    dba_stats st{};
    double seconds = 0.0;
    for (int it = 0; it < max_iters; ++it) {
      // one iteration and the stopping test's metrics pass (rmse_gt only; the full statistics
      // are evaluated once at the end), one graph launch when graphs are on
      DBA_CUDA(cudaEventRecord(ctx->ev0, ctx->stream), "event");
      if (ctx->cfg.use_graph) {
        dba_status s = ensure_graph(ctx, true);
        if (s != DBA_OK) return s;
        DBA_CUDA(cudaGraphLaunch(ctx->graph_until, ctx->stream), "graph launch");
        ctx->cur ^= 1;
        ctx->pending = 1;
        ctx->iters += 1;
      } else {
        dba_status s = run_iterations(ctx, 1);
        if (s != DBA_OK) return s;
        DBA_CUDA(dba::launch_metrics(ctx->P, ctx->prm, ctx->fp32, ctx->cur, ctx->pending, ctx->stream, true),
                 "metrics");
      }
      DBA_CUDA(cudaEventRecord(ctx->ev1, ctx->stream), "event");
      double h[8];
      DBA_CUDA(cudaMemcpyAsync(h, ctx->P.metric_out, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "metrics copy");
      dba_status s = check_device_flags(ctx);  // one synchronisation for both reads
      if (s != DBA_OK) return s;
      float ms = 0.f;
      DBA_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1), "event");
      seconds += ms * 1e-3;
      st.rmse_gt = h[7] > 0 ? std::sqrt(h[2] / h[7]) : 0.0;
      if (st.rmse_gt <= target_rmse_gt) break;
    }
    {
      dba_status s = read_metrics(ctx, &st, seconds);
      if (s != DBA_OK) return s;
    }
    if (stats) *stats = st;
    return DBA_OK;
  });
}

dba_status dba_evaluate(dba_ctx* ctx, dba_stats* stats) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx || !stats) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_evaluate before dba_set_observations");
    return read_metrics(ctx, stats, 0.0);
  });
}

dba_status dba_get_params(dba_ctx* ctx, double* cams, double* pts) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_get_params before dba_set_observations");
    cudaStream_t st = ctx->stream;
    std::vector<double> X(3 * (size_t)ctx->n_pts);
    if (cams)
      DBA_CUDA(cudaMemcpyAsync(cams, ctx->P.Y[ctx->cur], 6 * (size_t)ctx->n_cams * sizeof(double),
                               cudaMemcpyDeviceToHost, st), "read cameras");
    if (pts)
      DBA_CUDA(cudaMemcpyAsync(X.data(), ctx->P.X[ctx->cur], X.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
               "read points");
    DBA_CUDA(cudaStreamSynchronize(st), "get_params");
    if (pts)
      for (int k = 0; k < ctx->n_pts; ++k)
        for (int c = 0; c < 3; ++c) pts[3 * (size_t)ctx->pt_perm[k] + c] = X[3 * (size_t)k + c];
    return DBA_OK;
  });
}

dba_status dba_get_state(dba_ctx* ctx, double* copies, double* duals) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_get_state before dba_set_observations");
    cudaStream_t st = ctx->stream;
    if (ctx->pending) {
      DBA_CUDA(dba::launch_settle(ctx->P, ctx->fp32, ctx->cur, st), "settle");
      const int zero = 0;
      DBA_CUDA(cudaMemcpyAsync(&ctx->P.ctl->pending, &zero, sizeof zero, cudaMemcpyHostToDevice, st), "settle");
      DBA_CUDA(cudaStreamSynchronize(st), "settle");
      ctx->pending = 0;
    }
    const long long l = ctx->n_obs;
    const int m = ctx->n_cams, n = ctx->n_pts;
    std::vector<double> X(3 * (size_t)n), Y(6 * (size_t)m), del(9 * (size_t)l), a(9 * (size_t)l);
    DBA_CUDA(cudaMemcpyAsync(X.data(), ctx->P.X[ctx->cur], X.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "read");
    DBA_CUDA(cudaMemcpyAsync(Y.data(), ctx->P.Y[ctx->cur], Y.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "read");
    const size_t lp = (size_t)ctx->P.pitch;  // device rows pitched, host rows dense
    DBA_CUDA(cudaMemcpy2DAsync(a.data(), l * sizeof(double), ctx->P.adual, lp * sizeof(double), l * sizeof(double), 9,
                               cudaMemcpyDeviceToHost, st),
             "read");
    if (ctx->fp32) {
      std::vector<float> f(9 * (size_t)l);
      DBA_CUDA(cudaMemcpy2DAsync(f.data(), l * sizeof(float), ctx->P.delta, lp * sizeof(float), l * sizeof(float), 9,
                                 cudaMemcpyDeviceToHost, st),
               "read");
      DBA_CUDA(cudaStreamSynchronize(st), "get_state");
      for (size_t k = 0; k < f.size(); ++k) del[k] = f[k];
    } else {
      DBA_CUDA(cudaMemcpy2DAsync(del.data(), l * sizeof(double), ctx->P.delta, lp * sizeof(double), l * sizeof(double),
                                 9, cudaMemcpyDeviceToHost, st),
               "read");
      DBA_CUDA(cudaStreamSynchronize(st), "get_state");
    }
    for (long long o = 0; o < l; ++o) {
      const long long dst = ctx->perm[o];
      const size_t i = ctx->h_obs_pt[o], j = ctx->h_obs_cam[o];
      for (int c = 0; c < 9; ++c) {
        if (copies) copies[9 * dst + c] = (c < 3 ? X[3 * i + c] : Y[6 * j + c - 3]) + del[c * (size_t)l + o];
        if (duals) duals[9 * dst + c] = ctx->rho_of(c) * a[c * (size_t)l + o];
      }
    }
    return DBA_OK;
  });
}

dba_status dba_set_state(dba_ctx* ctx, const double* copies, const double* duals, const double* cams,
                         const double* pts, int64_t k) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_set_state before dba_set_observations");
    if (!copies || !duals || !cams || !pts) return ctx->fail(DBA_EINVAL, "dba_set_state: null array");
    if (k < 0) return ctx->fail(DBA_EINVAL, "dba_set_state: negative iteration count");
    if (!finite_all(copies, 9 * ctx->n_obs) || !finite_all(duals, 9 * ctx->n_obs) ||
        !finite_all(cams, 6 * (long long)ctx->n_cams) || !finite_all(pts, 3 * (long long)ctx->n_pts))
      return ctx->fail(DBA_EINVAL, "dba_set_state: non-finite value");
    const dba_status s = upload_state(ctx, cams, pts, copies, duals);
    if (s == DBA_OK) ctx->iters = k;
    return s;
  });
}

dba_status dba_inject_host_alloc_failure(int n) {
  if (n < 0) return DBA_EINVAL;
  dba::injected_host_alloc_failures() = n;
  return DBA_OK;
}

dba_status dba_build_layout(int32_t n_cams, int32_t n_pts, int64_t n_obs, const int32_t* pt_idx,
                            const int32_t* cam_idx, int tile_obs, int64_t* perm, int32_t* point,
                            int32_t* point_perm, int32_t* cam_rank, int64_t* tile_start, int64_t* n_tiles) {
  return dba::guarded(&g_create_error, [&]() -> dba_status {
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0 || n_obs > (int64_t)0x7fffffff || n_cams > dba::kCamMask ||
        !pt_idx || !cam_idx) {
      g_create_error = "dba_build_layout: sizes out of range or null index array";
      return DBA_EINVAL;
    }
    if (tile_obs != 64 && tile_obs != 128 && tile_obs != 256) {
      g_create_error = "dba_build_layout: tile_obs must be 64, 128 or 256";
      return DBA_EINVAL;
    }
    const long long bad = first_bad_index(pt_idx, cam_idx, n_obs, n_pts, n_cams);
    if (bad >= 0) {
      g_create_error = "dba_build_layout: observation " + std::to_string(bad) + " has an index out of range";
      return DBA_EINVAL;
    }
    HostLayout L;
    build_layout(n_cams, n_pts, n_obs, pt_idx, cam_idx, tile_obs, L);
    for (long long o = 0; o < n_obs; ++o) {
      if (perm) perm[o] = L.perm[o];
      if (point) point[o] = L.obs_pt[o];
      if (cam_rank) cam_rank[o] = (int32_t)((unsigned int)L.obs_cam_rank[o] >> 24);
    }
    if (point_perm)
      for (int k = 0; k < n_pts; ++k) point_perm[k] = L.pt_perm[k];
    if (tile_start) {
      for (size_t q = 0; q < L.tiles.size(); ++q) tile_start[q] = L.tiles[q].o0;
      tile_start[L.tiles.size()] = n_obs;
    }
    if (n_tiles) *n_tiles = (int64_t)L.tiles.size();
    return DBA_OK;
  });
}

dba_status dba_inject_copy_stall(dba_ctx* ctx, int on) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_inject_copy_stall before dba_set_observations");
    const unsigned int v = on ? 1u : 0u;
    DBA_CUDA(cudaMemcpyAsync(&ctx->P.ctl->inject, &v, sizeof v, cudaMemcpyHostToDevice, ctx->stream), "inject");
    DBA_CUDA(cudaStreamSynchronize(ctx->stream), "inject");
    return DBA_OK;
  });
}

dba_status dba_profile(dba_ctx* ctx, int n_iters, const char** names, double* ms, int* count) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx || !count) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_profile before dba_set_observations");
    if (n_iters <= 0 || *count < 2 || !names || !ms) return ctx->fail(DBA_EINVAL, "dba_profile: bad arguments");
    const int capacity = *count;
    std::vector<cudaEvent_t> ev(3 * (size_t)n_iters);
    for (auto& e : ev) DBA_CUDA(cudaEventCreate(&e), "event");
    cudaStream_t st = ctx->stream;
    std::vector<cudaEvent_t> evw(ctx->warm ? (size_t)n_iters : 0);
    for (auto& e : evw) DBA_CUDA(cudaEventCreate(&e), "event");
    for (int it = 0; it < n_iters; ++it) {
      if (ctx->warm) {
        DBA_CUDA(cudaEventRecord(evw[it], st), "event");
        DBA_CUDA(dba::launch_mlp_warmstart(ctx->P, ctx->prm, ctx->fp32, ctx->d_mlp_blob, ctx->d_mlp_params, st),
                 "warm start");
      }
      DBA_CUDA(cudaEventRecord(ev[3 * it], st), "event");
      DBA_CUDA(dba::launch_tile_iterate(ctx->P, ctx->tmaps, ctx->prm, ctx->fp32, st), "tile_iterate");
      DBA_CUDA(cudaEventRecord(ev[3 * it + 1], st), "event");
      DBA_CUDA(dba::launch_finalize(ctx->P, ctx->fp32, st), "finalize");
      DBA_CUDA(cudaEventRecord(ev[3 * it + 2], st), "event");
    }
    ctx->cur ^= (n_iters & 1);
    ctx->pending = 1;
    ctx->iters += n_iters;
    dba_status s = check_device_flags(ctx);
    double t0 = 0, t1 = 0, tw = 0;
    for (int it = 0; it < n_iters && s == DBA_OK; ++it) {
      float a = 0, b = 0, c = 0;
      cudaEventElapsedTime(&a, ev[3 * it], ev[3 * it + 1]);
      cudaEventElapsedTime(&b, ev[3 * it + 1], ev[3 * it + 2]);
      if (ctx->warm) cudaEventElapsedTime(&c, evw[it], ev[3 * it]);
      t0 += a;
      t1 += b;
      tw += c;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (auto& e : evw) cudaEventDestroy(e);
    if (s != DBA_OK) return s;
    names[0] = "tile_iterate";
    ms[0] = t0 / n_iters;
    names[1] = "finalize";
    ms[1] = t1 / n_iters;
    *count = 2;
    if (ctx->warm && capacity >= 3) {
      names[2] = "mlp_warm_start";
      ms[2] = tw / n_iters;
      *count = 3;
    }
    return DBA_OK;
  });
}

dba_status dba_layout(dba_ctx* ctx, int64_t* out, int* count) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx || !out || !count) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_layout before dba_set_observations");
    const int64_t v[7] = {ctx->P.n_tiles, ctx->P.tile_obs, ctx->n_pseg, (int64_t)ctx->P.n_cam_slots,
                          (int64_t)ctx->P.n_split_pts, (int64_t)ctx->P.n_pt_slots, (int64_t)ctx->P.fin_threads};
    const int n = std::min(*count, 7);
    for (int k = 0; k < n; ++k) out[k] = v[k];
    *count = n;
    return DBA_OK;
  });
}

dba_status dba_evaluate_noalloc(const dba_config* cfg, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                                const int32_t* pt_idx, const int32_t* cam_idx, const double* z,
                                const double* cams, const double* pts, double* out, void* stream) {
  return dba::guarded(&g_create_error, [&]() -> dba_status {
    if (!cfg || !out || (n_obs > 0 && (!pt_idx || !cam_idx || !z || !cams || !pts))) {
      g_create_error = "dba_evaluate_noalloc: null pointer";
      return DBA_EINVAL;
    }
    if (n_obs < 0 || n_obs > (int64_t)DBA_NOALLOC_MAX_OBS || n_cams < 0 || n_pts < 0) {
      g_create_error = "dba_evaluate_noalloc: n_obs must lie in [0, " + std::to_string(DBA_NOALLOC_MAX_OBS) +
                       "] (the size of its fixed device scratch) and n_cams, n_pts must be >= 0";
      return DBA_EINVAL;
    }
    if (!(std::isfinite(cfg->focal) && cfg->focal > 0 && std::isfinite(cfg->cx) && std::isfinite(cfg->cy) &&
          cfg->loss >= 0 && cfg->loss <= 2 &&
          (cfg->loss == DBA_LOSS_L2 || (std::isfinite(cfg->loss_param) && cfg->loss_param > 0)) &&
          std::isfinite(cfg->eps_depth))) {
      g_create_error = "dba_evaluate_noalloc: invalid configuration (focal, principal point, loss, eps_depth)";
      return DBA_EINVAL;
    }
    const Params prm{cfg->focal, cfg->cx, cfg->cy, cfg->loss, cfg->loss_param, 1.0, 1.0, 1.0,
                     0, 1e-3, 0.0, cfg->eps_depth, 0.0, DBA_SOLVER_GN};
    const cudaError_t e = dba::launch_eval_noalloc(prm, n_obs, n_cams, n_pts, pt_idx, cam_idx, z, cams, pts, out,
                                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
      g_create_error = std::string("dba_evaluate_noalloc: ") + cudaGetErrorString(e);
      return DBA_ECUDA;
    }
    return DBA_OK;
  });
}

dba_status dba_set_scenes(dba_ctx* ctx, int32_t n_scenes, const int64_t* obs_off, const int32_t* cam_off,
                          const int32_t* pt_off) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_set_scenes before dba_set_observations");
    if (n_scenes <= 0 || !obs_off || !cam_off || !pt_off) return ctx->fail(DBA_EINVAL, "dba_set_scenes: bad arguments");
    if (obs_off[0] != 0 || cam_off[0] != 0 || pt_off[0] != 0 || obs_off[n_scenes] != ctx->n_obs ||
        cam_off[n_scenes] != ctx->n_cams || pt_off[n_scenes] != ctx->n_pts)
      return ctx->fail(DBA_EINVAL, "dba_set_scenes: offsets must start at 0 and end at n_obs, n_cams, n_pts");
    for (int sc = 0; sc < n_scenes; ++sc)
      if (obs_off[sc + 1] < obs_off[sc] || cam_off[sc + 1] < cam_off[sc] || pt_off[sc + 1] < pt_off[sc])
        return ctx->fail(DBA_EINVAL, "dba_set_scenes: offsets must be nondecreasing");
    // scene of every caller observation, checked against its camera and point
    std::vector<int> scene_caller(ctx->n_obs);
    std::vector<int> cam_scene(ctx->n_cams), pt_scene(ctx->n_pts);
    for (int sc = 0; sc < n_scenes; ++sc) {
      for (int64_t o = obs_off[sc]; o < obs_off[sc + 1]; ++o) scene_caller[o] = sc;
      for (int32_t j = cam_off[sc]; j < cam_off[sc + 1]; ++j) cam_scene[j] = sc;
      for (int32_t i = pt_off[sc]; i < pt_off[sc + 1]; ++i) pt_scene[i] = sc;
    }
    std::vector<int> scene_int(ctx->n_obs);
    for (long long o = 0; o < ctx->n_obs; ++o) {
      const long long src = ctx->perm[o];
      const int sc = scene_caller[src];
      if (cam_scene[ctx->h_obs_cam[o]] != sc || pt_scene[ctx->pt_perm[ctx->h_obs_pt[o]]] != sc)
        return ctx->fail(DBA_EINVAL, "dba_set_scenes: observation " + std::to_string(src) + " leaves its scene");
      scene_int[o] = sc;
    }
    const int* d = nullptr;
    DBA_CUDA(ctx->upload(&d, scene_int), "upload scenes");
    ctx->d_scene_of_obs = const_cast<int*>(d);
    DBA_CUDA(ctx->alloc(&ctx->d_scene_sums, 5 * (size_t)n_scenes), "alloc scene sums");
    DBA_CUDA(cudaStreamSynchronize(ctx->stream), "set_scenes");
    ctx->n_scenes = n_scenes;
    return DBA_OK;
  });
}

dba_status dba_scene_stats(dba_ctx* ctx, double* rmse_obs, double* rmse_gt, double* objective) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem || ctx->n_scenes == 0)
      return ctx->fail(DBA_ESTATE, "dba_scene_stats needs dba_set_observations and dba_set_scenes");
    cudaStream_t st = ctx->stream;
    std::vector<double> h(5 * (size_t)ctx->n_scenes);
    DBA_CUDA(cudaMemsetAsync(ctx->d_scene_sums, 0, h.size() * sizeof(double), st), "scene stats");
    DBA_CUDA(dba::launch_scene_metrics(ctx->P, ctx->prm, ctx->fp32, ctx->d_scene_of_obs, ctx->d_scene_sums, st),
             "scene stats");
    DBA_CUDA(cudaMemcpyAsync(h.data(), ctx->d_scene_sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
             "scene stats");
    DBA_CUDA(cudaStreamSynchronize(st), "scene stats");
    for (int sc = 0; sc < ctx->n_scenes; ++sc) {
      const double* v = &h[5 * (size_t)sc];
      if (rmse_obs) rmse_obs[sc] = v[3] > 0 ? std::sqrt(v[0] / v[3]) : 0.0;
      if (objective) objective[sc] = v[1];
      if (rmse_gt) rmse_gt[sc] = (ctx->has_gt && v[4] > 0) ? std::sqrt(v[2] / v[4]) : 0.0;
    }
    return DBA_OK;
  });
}

dba_status dba_mlp_harvest(dba_ctx* ctx, int64_t stride, int target_steps, float* feats, float* targets,
                           int64_t cap, int64_t* n_out) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_mlp_harvest before dba_set_observations");
    if (stride <= 0 || cap < 0 || target_steps < 0 || target_steps > 1000 || !feats || !targets || !n_out)
      return ctx->fail(DBA_EINVAL, "dba_mlp_harvest: bad arguments");
    const int64_t n = std::min<int64_t>(cap, (ctx->n_obs + stride - 1) / stride);
    DBA_CUDA(dba::launch_mlp_harvest(ctx->P, ctx->prm, ctx->fp32, ctx->pending, stride, n, target_steps, feats,
                                     targets, ctx->stream),
             "harvest");
    DBA_CUDA(cudaStreamSynchronize(ctx->stream), "harvest");
    *n_out = n;
    return DBA_OK;
  });
}

dba_status dba_set_warm_start(dba_ctx* ctx, const dba_mlp* mlp) {
  return dba::guarded(ctx ? &ctx->err : nullptr, [&]() -> dba_status {
    if (!ctx) return DBA_EINVAL;
    if (!ctx->has_problem) return ctx->fail(DBA_ESTATE, "dba_set_warm_start before dba_set_observations");
    ctx->drop_graphs();
    if (!mlp) {
      ctx->warm = false;
      ctx->P.mlp_start = nullptr;
      return DBA_OK;
    }
    std::vector<float> params(DBA_MLP_N_PARAMS);
    const dba_status ps = dba_mlp_get_params(mlp, params.data());
    if (ps != DBA_OK) return ctx->fail(ps, "dba_set_warm_start: cannot read the network");
    std::vector<unsigned char> blob;
    dba::mlp_make_blob(params.data(), blob);
    if (!ctx->d_mlp_blob) {
      DBA_CUDA(ctx->alloc(&ctx->d_mlp_blob, blob.size()), "warm start");
      DBA_CUDA(ctx->alloc(&ctx->d_mlp_params, params.size()), "warm start");
      char* p = nullptr;
      DBA_CUDA(ctx->alloc(&p, 9 * (size_t)ctx->P.pitch * (ctx->fp32 ? sizeof(float) : sizeof(double))), "warm start");
      ctx->P.mlp_start = p;
    }
    DBA_CUDA(cudaMemcpyAsync(ctx->d_mlp_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice, ctx->stream),
             "warm start");
    DBA_CUDA(cudaMemcpyAsync(ctx->d_mlp_params, params.data(), params.size() * sizeof(float), cudaMemcpyHostToDevice,
                             ctx->stream),
             "warm start");
    DBA_CUDA(cudaStreamSynchronize(ctx->stream), "warm start");
    ctx->warm = true;
    return DBA_OK;
  });
}

}  // extern "C"
