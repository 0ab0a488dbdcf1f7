// Batched RK4 stepping of many uneven grid patches (the single-GPU analogue
// of the block-structured AMR/multi-block grids the paper plans for, Sec. 4
// and Sec. 1.1; tile selection prior art, Sec. 2.6).
//
// A plan holds, for every patch, three stage buffers and its difference
// tables, a device table describing the patches, and one CUDA graph per
// step size. One RK4 step of all patches is one graph launch: four times
// (static ghost fill, [single-precision copy,] difference tables, fused
// stage), then a final ghost fill - every node a persistent kernel that walks
// a flat list of fixed-size tiles over all patches (grid-stride, so no device
// side waiting, no atomics, and a deterministic result).
//
// Tiles: each patch's interior is cut into tiles of tx*ty*tz points
// (tx*ty*tz = 128 = one CTA, one point per thread; ragged tiles at the
// patch edges idle their extra threads) or, for the "linear" shape, into runs
// of 128 consecutive points in x-fastest order. The shape per patch comes
// from an empirical autotuner: it times the fused stage kernel on one
// representative patch per size class with every candidate shape, and keeps
// the fastest in a process-wide cache keyed by (size class, order,
// precision). The per-point arithmetic is exactly the single-grid kernel's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/bssn.h"
#include "bssn_launch.h"
#include "bssn_patch.cuh"

using namespace bssn;

namespace {

constexpr int NSHAPES = 7;
// candidate tile shapes (tx, ty, tz); {0,0,0} = linear runs of 128 points
const int SHAPES[NSHAPES][3] = {{0, 0, 0}, {32, 4, 1}, {16, 8, 1}, {8, 8, 2}, {32, 2, 2}, {16, 4, 2}, {8, 4, 4}};

// size class of a patch for the tuning cache: bucket of its x extent and of
// its volume
int size_class(const bssn_grid_t& G) {
  const int xb = G.nx <= 24 ? 0 : (G.nx <= 48 ? 1 : 2);
  const long long v = (long long)G.nx * G.ny * G.nz;
  const int vb = v <= 32768 ? 0 : (v <= 262144 ? 1 : 2);
  return xb * 3 + vb;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune_cache;  // (class, order, prec) -> shape index

}  // namespace

struct bssn_plan {
  int np = 0;
  int order = 4;
  bssn_precision_t prec = BSSN_FP64;
  bssn_params_t params{};
  Gauge gz{};
  std::vector<PatchDev> host;
  PatchDev* dev = nullptr;
  long long* d_tile0 = nullptr;
  long long* d_ext0 = nullptr;
  long long* d_pad0 = nullptr;
  long long ntiles = 0, next = 0, npad = 0, points = 0;
  std::vector<void*> allocations;
  std::vector<int> shape;  // per patch
  int grid_stage = 0, grid_other = 0;
  // FP32-RHS form: the tiled kernels of bssn_stage32.cuh over a second table,
  // ordered by spacing so that each spacing's patches are one range
  std::vector<Patch32> host32;
  Patch32* dev32 = nullptr;
  long long* d_tile32 = nullptr;
  long long* d_pad32 = nullptr;
  long long* d_ext32 = nullptr;
  long long ntiles32 = 0, npad32 = 0, next32 = 0;
  struct Level {
    int p0, np;
    long long tbase, ntiles;
    Coef32 C;
  };
  std::vector<Level> levels;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double graph_dt = NAN;
  cudaStream_t cap = nullptr;
};

namespace {

cudaError_t plan_alloc(bssn_plan* pl, size_t bytes, void** out) {
  cudaError_t e = cudaMalloc(out, bytes);
  if (e == cudaSuccess) pl->allocations.push_back(*out);
  return e;
}

void plan_free(bssn_plan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  for (void* p : pl->allocations) cudaFree(p);
  pl->allocations.clear();
}

// (Re)compute tiles and offsets from the current shape choices and upload the
// patch table.
cudaError_t plan_upload(bssn_plan* pl) {
  const int H = pl->order / 2;
  std::vector<long long> t0(pl->np), e0(pl->np), p0(pl->np);
  long long nt = 0, ne = 0, npd = 0;
  for (int b = 0; b < pl->np; ++b) {
    PatchDev& D = pl->host[b];
    const int* s = SHAPES[pl->shape[b]];
    D.tx = s[0]; D.ty = s[1]; D.tz = s[2];
    const long long n = tiles_of(D.L, D.tx, D.ty, D.tz, &D.ntx, &D.nty);
    D.tile0 = t0[b] = nt;
    nt += n;
    D.ext0 = e0[b] = ne;
    ne += (long long)D.L.nx * (D.L.ny + 2 * H) * (D.L.nz + 2 * H);
    D.pad0 = p0[b] = npd;
    npd += (D.L.nx + 2LL * D.L.g) * (D.L.ny + 2LL * D.L.g) * (D.L.nz + 2LL * D.L.g);
  }
  pl->ntiles = nt;
  pl->next = ne;
  pl->npad = npd;
  cudaError_t e = cudaMemcpy(pl->dev, pl->host.data(), sizeof(PatchDev) * pl->np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_tile0, t0.data(), sizeof(long long) * pl->np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_ext0, e0.data(), sizeof(long long) * pl->np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_pad0, p0.data(), sizeof(long long) * pl->np, cudaMemcpyHostToDevice);
  return e;
}

template <int PO, typename R>
cudaError_t launch_stage_all(bssn_plan* pl, const RK& rk, int in, int out, long long ntiles, const PatchDev* dev,
                             const long long* tile0, int np, cudaStream_t s) {
  const unsigned int g = (unsigned int)std::max<long long>(1, std::min<long long>(pl->grid_stage, ntiles));
  kb_stage<PO, R><<<g, TILE_THREADS, 0, s>>>(dev, tile0, np, ntiles, pl->gz, rk, in, out);
  return cudaGetLastError();
}

cudaError_t stage_all(bssn_plan* pl, const RK& rk, int in, int out, long long ntiles, const PatchDev* dev,
                      const long long* tile0, int np, cudaStream_t s) {
  const bool f64 = pl->prec == BSSN_FP64;
  if (pl->order == 4)
    return f64 ? launch_stage_all<4, double>(pl, rk, in, out, ntiles, dev, tile0, np, s)
               : launch_stage_all<4, float>(pl, rk, in, out, ntiles, dev, tile0, np, s);
  return f64 ? launch_stage_all<8, double>(pl, rk, in, out, ntiles, dev, tile0, np, s)
             : launch_stage_all<8, float>(pl, rk, in, out, ntiles, dev, tile0, np, s);
}

cudaError_t other_all(bssn_plan* pl, int kind, int which, cudaStream_t s) {
  const unsigned int g = (unsigned int)pl->grid_other;
  if (kind == 0) {
    kb_fill<<<g, 256, 0, s>>>(pl->dev, pl->d_pad0, pl->np, pl->npad, which);
  } else if (kind == 1) {
    kb_to_f32<<<g, 256, 0, s>>>(pl->dev, pl->d_pad0, pl->np, pl->npad, which);
  } else {
    const bool f64 = pl->prec == BSSN_FP64;
    if (pl->order == 4) {
      if (f64) kb_diffs<4, double><<<g, 256, 0, s>>>(pl->dev, pl->d_ext0, pl->np, pl->next, which);
      else kb_diffs<4, float><<<g, 256, 0, s>>>(pl->dev, pl->d_ext0, pl->np, pl->next, which);
    } else {
      if (f64) kb_diffs<8, double><<<g, 256, 0, s>>>(pl->dev, pl->d_ext0, pl->np, pl->next, which);
      else kb_diffs<8, float><<<g, 256, 0, s>>>(pl->dev, pl->d_ext0, pl->np, pl->next, which);
    }
  }
  return cudaGetLastError();
}

// One FP32-RHS stage of all patches with the tiled kernels: single-precision
// copy of the stage input, D_x / D_y tables, then one stage launch per
// spacing.
cudaError_t stage32_all(bssn_plan* pl, const RK& rk, int in, int out, cudaStream_t s) {
  const int g = pl->grid_other;
  cudaError_t e = launch_to_f32t_batch(pl->dev32, pl->d_pad32, pl->np, pl->npad32, in, g, s);
  if (e == cudaSuccess)
    e = pl->order == 4 ? launch_d1tab32_batch<4>(pl->dev32, pl->d_ext32, pl->np, pl->next32, g, s)
                       : launch_d1tab32_batch<8>(pl->dev32, pl->d_ext32, pl->np, pl->next32, g, s);
  for (const auto& lv : pl->levels) {
    if (e != cudaSuccess) break;
    e = pl->order == 4 ? launch_stage32_batch<4>(pl->dev32, pl->d_tile32, lv.p0, lv.np, lv.tbase, lv.ntiles, lv.C,
                                                 pl->gz, rk, in, out, s)
                       : launch_stage32_batch<8>(pl->dev32, pl->d_tile32, lv.p0, lv.np, lv.tbase, lv.ntiles, lv.C,
                                                 pl->gz, rk, in, out, s);
  }
  return e;
}

// The launch sequence of one RK4 step (captured into the graph).
cudaError_t enqueue_step(bssn_plan* pl, double dt, cudaStream_t s) {
  const int ins[4] = {0, 1, 2, 1};
  const int outs[4] = {1, 2, 1, 0};
  cudaError_t e = cudaSuccess;
  for (int st = 0; st < 4 && e == cudaSuccess; ++st) {
    if (pl->prec == BSSN_FP32_RHS) {
      e = other_all(pl, 0, ins[st], s);
      if (e == cudaSuccess) e = stage32_all(pl, make_rk(st, dt), ins[st], outs[st], s);
      continue;
    }
    e = other_all(pl, 0, ins[st], s);
    if (e == cudaSuccess && pl->prec == BSSN_FP32_RHS) e = other_all(pl, 1, ins[st], s);
    if (e == cudaSuccess) e = other_all(pl, 2, ins[st], s);
    if (e == cudaSuccess) e = stage_all(pl, make_rk(st, dt), ins[st], outs[st], pl->ntiles, pl->dev, pl->d_tile0,
                                        pl->np, s);
  }
  if (e == cudaSuccess) e = other_all(pl, 0, 0, s);
  return e;
}

// Time the fused stage on patch b alone with tile shape `shape`.
float time_shape(bssn_plan* pl, int b, int shape, cudaStream_t s, cudaError_t* err) {
  PatchDev D = pl->host[b];
  const int* sh = SHAPES[shape];
  D.tx = sh[0]; D.ty = sh[1]; D.tz = sh[2];
  D.tile0 = 0;
  const long long nt = tiles_of(D.L, D.tx, D.ty, D.tz, &D.ntx, &D.nty);
  // a one-entry table at the end of the plan's device table scratch
  PatchDev* d1 = pl->dev + pl->np;
  long long* t1 = pl->d_tile0 + pl->np;
  long long zero = 0;
  *err = cudaMemcpy(d1, &D, sizeof(PatchDev), cudaMemcpyHostToDevice);
  if (*err == cudaSuccess) *err = cudaMemcpy(t1, &zero, sizeof(long long), cudaMemcpyHostToDevice);
  if (*err != cudaSuccess) return 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const RK rk = make_rk(0, 0.0);  // stage 0 with dt = 0 leaves the state unchanged
  float best = 1e30f;
  for (int rep = 0; rep < 3 && *err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    *err = stage_all(pl, rk, 0, 1, nt, d1, t1, 1, s);
    cudaEventRecord(e1, s);
    if (*err == cudaSuccess) *err = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

namespace bssn {
cudaError_t bounds_take_batch(unsigned long long* out) { return bounds_take_local(out); }
}  // namespace bssn

extern "C" {

bssn_status_t bssn_plan_create(bssn_plan_t** out, const bssn_block_t* blocks, int nblocks,
                               const bssn_params_t* params, bssn_precision_t prec, int autotune) {
  if (!out || !blocks || nblocks < 1 || nblocks > (1 << 20) || !params) return BSSN_ERR_INVALID_ARG;
  if (prec != BSSN_FP64 && prec != BSSN_FP32_RHS) return BSSN_ERR_INVALID_ARG;
  *out = nullptr;
  for (int b = 0; b < nblocks; ++b) {
    const bssn_block_t& B = blocks[b];
    if (bssn_work_bytes(&B.grid, params, prec) == 0) return BSSN_ERR_INVALID_ARG;
    if (!B.state || !B.ghost_src || ((uintptr_t)B.state & 15) || ((uintptr_t)B.ghost_src & 15))
      return BSSN_ERR_INVALID_ARG;
    if (B.state == B.ghost_src) return BSSN_ERR_INVALID_ARG;
  }
  bssn_plan* pl = new (std::nothrow) bssn_plan;
  if (!pl) return BSSN_ERR_NOMEM;
  pl->np = nblocks;
  pl->order = params->fd_order;
  pl->prec = prec;
  pl->params = *params;
  pl->gz = make_gauge(*params);
  pl->host.resize(nblocks);
  pl->shape.assign(nblocks, 0);
  cudaError_t e = cudaSuccess;
  const int H = pl->order / 2;
  for (int b = 0; b < nblocks && e == cudaSuccess; ++b) {
    const bssn_block_t& B = blocks[b];
    PatchDev& D = pl->host[b];
    std::memset((void*)&D, 0, sizeof(D));
    D.L = make_layout(B.grid);
    D.buf[0] = B.state;
    D.ghost = B.ghost_src;
    const size_t n = (size_t)NV * B.grid.var_stride;
    void* p = nullptr;
    e = plan_alloc(pl, 3 * n * sizeof(double), &p);
    if (e != cudaSuccess) break;
    D.buf[1] = (double*)p;
    D.buf[2] = D.buf[1] + n;
    D.buf[3] = D.buf[2] + n;
    // stage buffers start as a copy of the state so their ghosts are defined
    e = cudaMemcpy(D.buf[1], B.state, n * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D.buf[2], B.state, n * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemset(D.buf[3], 0, n * sizeof(double));
    if (e != cudaSuccess) break;
    if (prec == BSSN_FP64) {
      const size_t tab = (size_t)NM * H * B.grid.var_stride;
      e = plan_alloc(pl, 2 * tab * sizeof(double), &p);
      if (e != cudaSuccess) break;
      D.dX = p;
      D.dY = (char*)p + tab * sizeof(double);
    }
    if (pl->order == 4) {
      D.c64 = make_coef<4, double>(B.grid, params->ko_eps);
      D.c32 = make_coef<4, float>(B.grid, params->ko_eps);
    } else {
      D.c64 = make_coef<8, double>(B.grid, params->ko_eps);
      D.c32 = make_coef<8, float>(B.grid, params->ko_eps);
    }
    pl->points += D.L.npts;
  }
  void* p = nullptr;
  // FP32-RHS: per patch a single-precision copy and tables in Layout32, and
  // the tiled kernels' table, sorted by spacing (one stage launch each)
  if (e == cudaSuccess && prec == BSSN_FP32_RHS) {
    std::vector<int> ord(nblocks);
    for (int b = 0; b < nblocks; ++b) ord[b] = b;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const bssn_grid_t &A = blocks[a].grid, &Bg = blocks[b].grid;
      return std::make_tuple(A.dx, A.dy, A.dz) < std::make_tuple(Bg.dx, Bg.dy, Bg.dz);
    });
    pl->host32.resize(nblocks);
    std::vector<long long> t0(nblocks), q0(nblocks), x0(nblocks);
    long long nt = 0, nq = 0, nx = 0;
    for (int i = 0; i < nblocks && e == cudaSuccess; ++i) {
      const int b = ord[i];
      const bssn_grid_t& G = blocks[b].grid;
      const Layout32 L32 = make_layout32(G);
      e = plan_alloc(pl, (size_t)(NV + 2 * NM) * L32.vs * sizeof(float), &p);
      if (e != cudaSuccess) break;
      float* f32 = (float*)p;
      float* tab = f32 + (size_t)NV * L32.vs;
      Patch32& Q = pl->host32[i];
      std::memset((void*)&Q, 0, sizeof(Q));
      const bool ok = pl->order == 4 ? make_patch32<4>(&Q, G, params->ko_eps, pl->host[b].buf, f32, tab)
                                     : make_patch32<8>(&Q, G, params->ko_eps, pl->host[b].buf, f32, tab);
      if (!ok) {
        e = cudaErrorInvalidValue;
        break;
      }
      Q.tile0 = t0[i] = nt;
      nt += (long long)Q.ntx * Q.nty * ((G.nz + 3) / 4);
      Q.pad0 = q0[i] = nq;
      nq += (G.nx + 2LL * G.ghost) * (G.ny + 2LL * G.ghost) * (G.nz + 2LL * G.ghost);
      Q.ext0 = x0[i] = nx;
      nx += (long long)G.nx * (G.ny + 2 * H) * (G.nz + 2 * H);
      if (i == 0 || G.dx != blocks[ord[i - 1]].grid.dx || G.dy != blocks[ord[i - 1]].grid.dy ||
          G.dz != blocks[ord[i - 1]].grid.dz)
        pl->levels.push_back({i, 0, Q.tile0, 0, Q.C});
      pl->levels.back().np += 1;
      pl->levels.back().ntiles = nt - pl->levels.back().tbase;
    }
    pl->ntiles32 = nt;
    pl->npad32 = nq;
    pl->next32 = nx;
    if (e == cudaSuccess) e = plan_alloc(pl, sizeof(Patch32) * nblocks, &p);
    if (e == cudaSuccess) pl->dev32 = (Patch32*)p;
    if (e == cudaSuccess) e = plan_alloc(pl, 3 * sizeof(long long) * nblocks, &p);
    if (e == cudaSuccess) {
      pl->d_tile32 = (long long*)p;
      pl->d_pad32 = pl->d_tile32 + nblocks;
      pl->d_ext32 = pl->d_pad32 + nblocks;
      e = cudaMemcpy(pl->dev32, pl->host32.data(), sizeof(Patch32) * nblocks, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_tile32, t0.data(), sizeof(long long) * nblocks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_pad32, q0.data(), sizeof(long long) * nblocks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pl->d_ext32, x0.data(), sizeof(long long) * nblocks, cudaMemcpyHostToDevice);
    // the tiles are the tiled kernel's 8 x 4 x 4 (shape 6)
    pl->shape.assign(nblocks, 6);
    if (e == cudaSuccess) e = pl->order == 4 ? stage32_batch_init<4>() : stage32_batch_init<8>();
  }
  if (e == cudaSuccess) e = plan_alloc(pl, sizeof(PatchDev) * (nblocks + 1), &p);
  if (e == cudaSuccess) pl->dev = (PatchDev*)p;
  if (e == cudaSuccess) e = plan_alloc(pl, sizeof(long long) * (nblocks + 1), &p);
  if (e == cudaSuccess) pl->d_tile0 = (long long*)p;
  if (e == cudaSuccess) e = plan_alloc(pl, sizeof(long long) * nblocks, &p);
  if (e == cudaSuccess) pl->d_ext0 = (long long*)p;
  if (e == cudaSuccess) e = plan_alloc(pl, sizeof(long long) * nblocks, &p);
  if (e == cudaSuccess) pl->d_pad0 = (long long*)p;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
  // persistent grids: resident CTAs per SM x SMs
  int dev = 0, sms = 0, occ = 1;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (pl->order == 4)
      e = prec == BSSN_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<4, double>, TILE_THREADS, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<4, float>, TILE_THREADS, 0);
    else
      e = prec == BSSN_FP64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<8, double>, TILE_THREADS, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_stage<8, float>, TILE_THREADS, 0);
  }
  pl->grid_stage = std::max(1, occ) * std::max(1, sms);
  pl->grid_other = 8 * std::max(1, sms);
  if (e == cudaSuccess) e = plan_upload(pl);

  // empirical tile-shape tuning, per size class, cached per process; the
  // stage is timed on real difference tables of the initial state
  // (the FP32-RHS form runs the tiled kernel, whose tile is fixed)
  if (e == cudaSuccess && autotune && prec == BSSN_FP64) {
    e = other_all(pl, 0, 0, pl->cap);
    if (e == cudaSuccess) e = other_all(pl, 2, 0, pl->cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl->cap);
  }
  if (e == cudaSuccess && autotune && prec == BSSN_FP64) {
    std::map<int, int> rep;  // class -> representative patch (largest)
    for (int b = 0; b < nblocks; ++b) {
      const int c = size_class(blocks[b].grid);
      auto it = rep.find(c);
      if (it == rep.end() || pl->host[b].L.npts > pl->host[it->second].L.npts) rep[c] = b;
    }
    for (auto& kv : rep) {
      const auto key = std::make_tuple(kv.first, pl->order, (int)prec);
      int best = -1;
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
      }
      if (best < 0) {
        float tbest = 1e30f;
        for (int sidx = 0; sidx < NSHAPES && e == cudaSuccess; ++sidx) {
          const float t = time_shape(pl, kv.second, sidx, pl->cap, &e);
          if (t < tbest) { tbest = t; best = sidx; }
        }
        if (e != cudaSuccess) break;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
      }
      for (int b = 0; b < nblocks; ++b)
        if (size_class(blocks[b].grid) == kv.first) pl->shape[b] = best;
    }
    if (e == cudaSuccess) e = plan_upload(pl);
  }
  if (e != cudaSuccess) {
    plan_free(pl);
    delete pl;
    return e == cudaErrorMemoryAllocation ? BSSN_ERR_NOMEM : BSSN_ERR_CUDA;
  }
  *out = pl;
  return BSSN_OK;
}

bssn_status_t bssn_batch_step(bssn_plan_t* pl, double dt, void* stream) {
  if (!pl || !std::isfinite(dt)) return BSSN_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (!pl->exec || pl->graph_dt != dt) {
    if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
    if (pl->graph) { cudaGraphDestroy(pl->graph); pl->graph = nullptr; }
    e = cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_step(pl, dt, pl->cap);
      e = cudaStreamEndCapture(pl->cap, &pl->graph);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    if (e != cudaSuccess) return BSSN_ERR_CUDA;
    pl->graph_dt = dt;
  }
  e = cudaGraphLaunch(pl->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? BSSN_OK : BSSN_ERR_CUDA;
}

bssn_status_t bssn_plan_info(const bssn_plan_t* pl, long long* points, long long* tiles, int* shapes) {
  if (!pl) return BSSN_ERR_INVALID_ARG;
  if (points) *points = pl->points;
  if (tiles) *tiles = pl->ntiles;
  if (shapes)
    for (int b = 0; b < pl->np; ++b) shapes[b] = pl->shape[b];
  return BSSN_OK;
}

bssn_status_t bssn_plan_destroy(bssn_plan_t* pl) {
  if (!pl) return BSSN_ERR_INVALID_ARG;
  plan_free(pl);
  delete pl;
  return BSSN_OK;
}

}  // extern "C"
