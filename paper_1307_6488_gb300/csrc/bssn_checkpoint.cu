// Checkpoint and resume of one evolved grid: the padded FP64 state (all 24
// variables, ghosts included, var_stride apart) with the grid, the evolution
// parameters, the time and the step count, in one file. Host memory only:
// the caller copies the state off the device before writing and back after
// reading, so a resumed evolution continues from exactly the same bits.
// The file is written under a temporary name, flushed to disk and renamed
// over `path` only once every write succeeded, so a failed or interrupted
// write leaves the previous checkpoint at `path` intact.
//
// File layout (native little-endian, as on both host architectures):
//   "BSSNCKP1", uint32 byte-order mark 0x01020304, uint32 format version 1,
//   int32 nx, ny, nz, ghost; double dx, dy, dz; int64 var_stride;
//   int32 fd_order; double ko_eps; int32 lapse, shift; double shift_coeff,
//   eta; int32 advect_gauge; double t; int64 step; int64 data doubles;
//   uint64 FNV-1a hash of the data bytes; then the data.
#include <unistd.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bssn.h"
#include "bssn_launch.h"

namespace {

constexpr char MAGIC[8] = {'B', 'S', 'S', 'N', 'C', 'K', 'P', '1'};
constexpr uint32_t BOM = 0x01020304u;
constexpr uint32_t VERSION = 1;
constexpr int NVARS = 24;

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// a grid a file may describe (bounded, so that no size computation overflows)
bool grid_valid(const bssn_grid_t& G) {
  const int lim = 1 << 20;
  if (G.nx < 1 || G.ny < 1 || G.nz < 1 || G.nx > lim || G.ny > lim || G.nz > lim) return false;
  if (G.ghost < 0 || G.ghost > 64) return false;
  if (!(G.dx > 0) || !(G.dy > 0) || !(G.dz > 0)) return false;
  if (!std::isfinite(G.dx) || !std::isfinite(G.dy) || !std::isfinite(G.dz)) return false;
  const long long pad = ((long long)G.nx + 2LL * G.ghost) * ((long long)G.ny + 2LL * G.ghost) *
                        ((long long)G.nz + 2LL * G.ghost);
  return pad <= (1LL << 44) && G.var_stride >= pad && G.var_stride <= (1LL << 44) && G.var_stride % 2 == 0;
}

// sequential writer / reader of plain fields
struct Out {
  std::vector<unsigned char> b;
  template <typename T>
  void put(const T& v) {
    const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
    b.insert(b.end(), p, p + sizeof(T));
  }
};

struct In {
  const unsigned char* p;
  size_t n, at = 0;
  template <typename T>
  bool get(T* v) {
    if (at + sizeof(T) > n) return false;
    std::memcpy(v, p + at, sizeof(T));
    at += sizeof(T);
    return true;
  }
};

}  // namespace

extern "C" {

bssn_status_t bssn_checkpoint_write(const char* path, const bssn_grid_t* grid, const bssn_params_t* params, double t,
                                    long long step, const double* state) {
  if (!path || !grid || !params || !state || !grid_valid(*grid) || !std::isfinite(t)) return BSSN_ERR_INVALID_ARG;
  if (!bssn::grid_params_valid(grid, params)) return BSSN_ERR_INVALID_ARG;
  const long long ndata = NVARS * grid->var_stride;
  Out h;
  h.b.insert(h.b.end(), MAGIC, MAGIC + 8);
  h.put(BOM);
  h.put(VERSION);
  h.put((int32_t)grid->nx);
  h.put((int32_t)grid->ny);
  h.put((int32_t)grid->nz);
  h.put((int32_t)grid->ghost);
  h.put(grid->dx);
  h.put(grid->dy);
  h.put(grid->dz);
  h.put((int64_t)grid->var_stride);
  h.put((int32_t)params->fd_order);
  h.put(params->ko_eps);
  h.put((int32_t)params->lapse);
  h.put((int32_t)params->shift);
  h.put(params->shift_coeff);
  h.put(params->eta);
  h.put((int32_t)params->advect_gauge);
  h.put(t);
  h.put((int64_t)step);
  h.put((int64_t)ndata);
  h.put(fnv1a(reinterpret_cast<const unsigned char*>(state), (size_t)ndata * sizeof(double)));
  const std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return BSSN_ERR_INVALID_ARG;
  bool ok = std::fwrite(h.b.data(), 1, h.b.size(), f) == h.b.size();
  ok = ok && std::fwrite(state, sizeof(double), (size_t)ndata, f) == (size_t)ndata;
  ok = ok && std::fflush(f) == 0 && fsync(fileno(f)) == 0;
  ok = (std::fclose(f) == 0) && ok;
  ok = ok && std::rename(tmp.c_str(), path) == 0;
  if (!ok) std::remove(tmp.c_str());
  return ok ? BSSN_OK : BSSN_ERR_INVALID_ARG;
}

bssn_status_t bssn_checkpoint_read(const char* path, bssn_grid_t* grid, bssn_params_t* params, double* t,
                                   long long* step, double* state, unsigned long long capacity) {
  if (!path || !grid || !params || !t || !step) return BSSN_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return BSSN_ERR_INVALID_ARG;
  // the fixed-size header written above: magic, mark and version (16),
  // sizes (16), spacing (24), var_stride (8), parameters (4 + 8 + 8 + 16 +
  // 4), t, step, data count and hash (32): 136 bytes
  constexpr size_t HEAD = 16 + 16 + 24 + 8 + 40 + 32;
  unsigned char buf[HEAD];
  if (std::fread(buf, 1, HEAD, f) != HEAD) {
    std::fclose(f);
    return BSSN_ERR_INVALID_ARG;
  }
  In in{buf, HEAD};
  char magic[8];
  uint32_t bom = 0, version = 0;
  int32_t nx, ny, nz, ghost, order, lapse, shift, adv;
  double dx, dy, dz, eps, coeff, eta, time;
  int64_t vs, nstep, ndata;
  uint64_t hash;
  bool ok = in.get(&magic) && in.get(&bom) && in.get(&version) && in.get(&nx) && in.get(&ny) && in.get(&nz) &&
            in.get(&ghost) && in.get(&dx) && in.get(&dy) && in.get(&dz) && in.get(&vs) && in.get(&order) &&
            in.get(&eps) && in.get(&lapse) && in.get(&shift) && in.get(&coeff) && in.get(&eta) && in.get(&adv) &&
            in.get(&time) && in.get(&nstep) && in.get(&ndata) && in.get(&hash);
  ok = ok && std::memcmp(magic, MAGIC, 8) == 0 && bom == BOM && version == VERSION;
  bssn_grid_t G{nx, ny, nz, ghost, dx, dy, dz, (long long)vs};
  bssn_params_t Pm{order, eps, lapse, shift, coeff, eta, adv};
  ok = ok && grid_valid(G) && ndata == NVARS * vs;
  // the parameters must be ones every stepping entry point accepts, and t finite
  ok = ok && bssn::grid_params_valid(&G, &Pm) && std::isfinite(time);
  if (ok && state) {
    ok = capacity >= (unsigned long long)ndata &&
         std::fread(state, sizeof(double), (size_t)ndata, f) == (size_t)ndata &&
         fnv1a(reinterpret_cast<const unsigned char*>(state), (size_t)ndata * sizeof(double)) == hash;
  }
  std::fclose(f);
  if (!ok) return BSSN_ERR_INVALID_ARG;
  *grid = G;
  params->fd_order = order;
  params->ko_eps = eps;
  params->lapse = lapse;
  params->shift = shift;
  params->shift_coeff = coeff;
  params->eta = eta;
  params->advect_gauge = adv;
  *t = time;
  *step = nstep;
  return BSSN_OK;
}

}  // extern "C"
