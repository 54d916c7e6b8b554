// fwi_api.cu -- host side of libfwi: context, checkpoint planner, point lists,
// TMA descriptors and the C ABI entry points declared in fwi.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fwi_internal.cuh"

using namespace fwi;

// ---------------------------------------------------------------- helpers --

namespace {

cudaError_t g_last_cuda_error = cudaSuccess;

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) {                       \
      g_last_cuda_error = e_;                      \
      return FWI_ERR_CUDA;                         \
    }                                              \
  } while (0)

constexpr double A8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
constexpr double RHO8 = 205.0 / 72.0 + 2.0 * (8.0 / 5.0 + 1.0 / 5.0 + 8.0 / 315.0 + 1.0 / 560.0);

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Checkpoint plan: snapshots p^0..p^{nt-1} are grouped in segments of K.
// The first forward pass keeps checkpoint pairs (p^{jK-1}, p^{jK}) for the
// segments 1..jL-1 and the snapshots of the last segment jL directly; the
// reverse pass recomputes every other segment from its checkpoint into the
// snapshot buffer.  Slot map: 0 zero field, 1..3 forward ring, 4..6 adjoint
// ring, then 2 (jL-1) checkpoint slots, then K snapshot slots.
struct Plan {
  int nt = 0, K = 0, jL = 0;
  long long recompute = 0;
  int slots = 0;
  static constexpr int ZERO = 0, RING = 1, QR = 4, CK0 = 7;
  int seg0() const { return CK0 + 2 * std::max(jL - 1, 0); }
  int fslot(int m) const {  // slot of p^m during the first forward pass
    if (m <= 0) return ZERO;
    if (m >= nt) return RING + m % 3;
    if (m >= jL * K) return seg0() + (m - jL * K);
    if ((m + 1) % K == 0) {
      const int j = (m + 1) / K;
      if (j >= 1 && j <= jL - 1) return CK0 + 2 * (j - 1);
    }
    if (m % K == 0) {
      const int j = m / K;
      if (j >= 1 && j <= jL - 1) return CK0 + 2 * (j - 1) + 1;
    }
    return RING + m % 3;
  }
  int rslot(int j, int m) const {  // slot of p^m while segment j < jL is recomputed
    if (m == j * K - 1) return j == 0 ? ZERO : CK0 + 2 * (j - 1);
    if (m == j * K) return j == 0 ? ZERO : CK0 + 2 * (j - 1) + 1;
    return seg0() + (m - j * K);
  }
  int snap(int j, int m) const { return j == jL ? fslot(m) : rslot(j, m); }
  int qslot(int k) const { return k > nt ? ZERO : QR + k % 3; }
};

bool make_plan(int nt, long long avail, Plan* out) {
  bool found = false;
  Plan best;
  for (int K = std::min(2, nt); K <= nt; K++) {
    Plan p;
    p.nt = nt;
    p.K = K;
    p.jL = (nt + K - 1) / K - 1;
    p.slots = Plan::CK0 + 2 * std::max(p.jL - 1, 0) + K;
    if (p.slots > avail) continue;
    p.recompute = (long long)p.jL * (K - 1);
    if (!found || p.recompute < best.recompute || (p.recompute == best.recompute && p.slots < best.slots)) {
      best = p;
      found = true;
    }
  }
  if (found) *out = best;
  return found;
}

constexpr int kTuneSteps = 6;  // steps per autotuner timing launch
constexpr int kMaxVariants = 32;  // step-kernel variants per direction (3D: five bits)
// 3D variant v runs all steps of a phase in one launch (bits 3 and 4 set)
inline bool multi_step3(int v) { return (v & 24) == 24; }
// Pinned staging buffers per kind (point lists, step descriptors), used in
// turn: an upload waits only for the copy issued kStaging uploads earlier,
// so the host can run that many gradient chunks ahead of the device before
// a call blocks.
constexpr int kStaging = 4;

// NVTX ranges (profiler annotations; no-ops when no tool is attached): one
// for the call, and inside it one for each phase in turn.  The destructor
// closes whatever is open, so early error returns stay balanced.
struct Ranges {
  int depth = 0;
  explicit Ranges(const char* call) { push(call); }
  void push(const char* name) {
    nvtxRangePushA(name);
    depth++;
  }
  void phase(const char* name) {
    if (depth > 1) {
      nvtxRangePop();
      depth--;
    }
    push(name);
  }
  ~Ranges() {
    while (depth-- > 0) nvtxRangePop();
  }
};

struct Entry {  // a point on the padded grid with a record column and amplitude
  int z, y, x, col;
  float amp;
};

}  // namespace

// ---------------------------------------------------------------- context --

struct fwi_ctx {
  fwi_grid g;
  Layout L;
  Coef K;
  int ns = 0, nr = 0, max_B = 0;
  std::vector<int> src_zyx, rec_zyx;  // padded coordinates
  int ntx = 0, ntz = 0, nty = 1, ntiles = 0;
  // tiles per tile shape: [0] the 2D tile or the 3D 64 x 16 tile, [1] the 3D
  // 64 x 8 pair tile (two supergathers per CTA); ntiles == ntiles_s[0]
  int ntiles_s[2] = {0, 0};
  double cell_volume = 1.0, vmax_cfl = 0.0;

  // device memory
  float* pool = nullptr;
  size_t pool_bytes = 0;
  int pool_B = -1;  // wavefields per slot of the current partition
  float* c = nullptr;      // [max_B][field]
  float* G = nullptr;      // [max_B][field]
  float* wav = nullptr;    // [nt]
  float* dpred = nullptr;  // [max_B][nt][nr]
  double* part = nullptr;  // [max_B][nblk]
  float* qsrc = nullptr;   // [max_B][nt][Emax]
  float* stmp = nullptr;   // [max_B][Emax]
  int* status = nullptr;
  int nblk = 0, Emax = 0;
  // receiver lists (shared by all wavefields): forward sampling, adjoint injection
  // per tile shape
  int* rec_off[2] = {};
  int2* rec_smp[2] = {};        // 2D sampling entries
  int4* rec_smp4[2] = {};       // 3D sampling entries (z in .z)
  int4* rec_inj[2] = {};        // adjoint injection entries (z in .w)
  // per-call lists
  unsigned char* dlist = nullptr;
  unsigned char* hlist[kStaging] = {};  // pinned staging, used in turn
  size_t list_bytes = 0;
  cudaEvent_t ev_list[kStaging] = {};
  int list_turn = 0;
  // profiling
  bool prof = false;
  cudaEvent_t ev[5] = {};
  long long launches[4] = {0, 0, 0, 0};
  Plan plan;
  long long slots_avail = 0;
  int chunk_samples = 0;
  bool last_was_gradient = false;
  float prof_ms[4] = {0.f, 0.f, 0.f, 0.f};
  // step-kernel variants: chosen per call shape by timing (autotune), or forced
  int var[2] = {-1, -1};
  int forced[2] = {-1, -1};
  int tuned_B = -1, tuned_nsg = -1;  // call shape the variants were tuned for
  int adj_pair = 0;  // tile shape of the 3D adjoint in the last tuned call (shape_adj)
  float tune_ms[2][kMaxVariants] = {};
  int* zero_off = nullptr;  // [ntiles+1] zeros: "no points in any tile"
  float* gtab = nullptr;    // gamma*dt per axis: z [nzp], y [nyp], x [nxp]
  // step descriptors of the current call, in launch order (device, pinned
  // staging, host copy), the autotuner's steps, and the per-item progress
  // flags of the multi-step 2D launches
  StepDesc* desc = nullptr;
  StepDesc* hdesc[kStaging] = {};
  size_t desc_cap = 0;
  cudaEvent_t ev_desc[kStaging] = {};
  int desc_turn = 0;
  std::vector<StepDesc> descs;
  StepDesc* tdesc = nullptr;
  int* done = nullptr;  // [max_B * ntiles]
};

namespace {

int check_grid(const fwi_grid* g) {
  if (!g || (g->ndim != 2 && g->ndim != 3)) return FWI_ERR_ARG;
  if (g->nz < 1 || g->nx < 1 || (g->ndim == 3 && g->ny < 1) || g->nb < 0 || g->nt < 1) return FWI_ERR_ARG;
  if (!(g->hz > 0) || !(g->hx > 0) || (g->ndim == 3 && !(g->hy > 0)) || !(g->dt > 0)) return FWI_ERR_ARG;
  if (!(g->sponge_vmax > 0) || !(g->sponge_R > 0 && g->sponge_R < 1)) return FWI_ERR_ARG;
  const double s = 1.0 / (g->hz * g->hz) + 1.0 / (g->hx * g->hx) + (g->ndim == 3 ? 1.0 / (g->hy * g->hy) : 0.0);
  if (g->sponge_vmax * g->sponge_vmax * g->dt * g->dt * RHO8 * s > 4.0) return FWI_ERR_CFL;
  return FWI_OK;
}

Layout make_layout(const fwi_grid* g) {
  Layout L;
  L.ndim = g->ndim;
  L.nz = g->nz;
  L.ny = g->ndim == 3 ? g->ny : 1;
  L.nx = g->nx;
  L.nb = g->nb;
  L.nzp = g->nz + 2 * g->nb;
  L.nyp = g->ndim == 3 ? g->ny + 2 * g->nb : 1;
  L.nxp = g->nx + 2 * g->nb;
  L.NZ = L.nzp + 2 * HALO;
  L.NY = g->ndim == 3 ? L.nyp + 2 * HALO : 1;
  L.SX = ((L.nxp + 2 * HALO) + 31) / 32 * 32;
  L.field = (long long)L.NZ * L.NY * L.SX;
  L.phys = (long long)L.nz * L.ny * L.nx;
  return L;
}

Coef make_coef(const fwi_grid* g) {
  Coef K;
  for (int k = 0; k < 5; k++) {
    K.cz[k] = (float)(A8[k] / (g->hz * g->hz));
    K.cx[k] = (float)(A8[k] / (g->hx * g->hx));
    K.cy[k] = g->ndim == 3 ? (float)(A8[k] / (g->hy * g->hy)) : 0.f;
  }
  double hmin = std::min(g->hz, g->hx);
  if (g->ndim == 3) hmin = std::min(hmin, g->hy);
  const double gmax = g->nb > 0 ? 3.0 * g->sponge_vmax * log(1.0 / g->sponge_R) / (2.0 * g->nb * hmin) : 0.0;
  K.gdt = (float)(gmax * g->dt);
  K.inv_nb = g->nb > 0 ? (float)(1.0 / g->nb) : 0.f;
  K.c0_2d = (float)(A8[0] / (g->hx * g->hx) + A8[0] / (g->hz * g->hz));
  K.c0_3d = g->ndim == 3 ? (float)(A8[0] / (g->hx * g->hx) + A8[0] / (g->hy * g->hy) + A8[0] / (g->hz * g->hz))
                         : 0.f;
  return K;
}

// Rows of a 3D wavefield tile for tile shape sh: 64 x 16, or 64 x 8 (pair tiles).
inline int tile_rows3(int sh) { return sh ? TY3 / 2 : TY3; }

// Tile of padded point (z, y, x) and its local index inside the tile.
// 2D tiles are 128 (x) x 32 or 128 x 24 (z); 3D tiles are 64 (x) x 16 or 64 x 8 (y) columns in z.
void tile_of(const fwi_ctx* C, const Entry& e, int sh, int* tile, int* local) {
  if (C->L.ndim == 3) {
    const int ty = tile_rows3(sh);
    *tile = (e.y / ty) * C->ntx + e.x / TX3;
    *local = (e.y % ty) * TX3 + (e.x % TX3);
  } else {
    const int tz = tile_rows2d(sh);
    *tile = (e.z / tz) * C->ntx + e.x / TX;
    *local = (e.z % tz) * TX + (e.x % TX);
  }
}

// Builds CSR offsets [nb_lists][ntiles+1] and entries for lists of points
// under tile shape sh.
template <typename Fill>
void build_csr(const fwi_ctx* C, const std::vector<std::vector<Entry>>& lists, int sh, int* off, Fill fill) {
  int pos = 0;
  const int nt = C->ntiles_s[sh];
  for (size_t b = 0; b < lists.size(); b++) {
    std::vector<std::pair<long long, int>> order;  // ((tile, z), index)
    for (size_t i = 0; i < lists[b].size(); i++) {
      int t, l;
      tile_of(C, lists[b][i], sh, &t, &l);
      order.push_back({(long long)t * (1LL << 32) + lists[b][i].z, (int)i});
    }
    std::stable_sort(order.begin(), order.end());
    size_t k = 0;
    for (int t = 0; t <= nt; t++) {
      off[b * (nt + 1) + t] = pos;
      if (t == nt) break;
      while (k < order.size() && (order[k].first >> 32) == t) {
        const Entry& e = lists[b][order[k].second];
        int tt, l;
        tile_of(C, e, sh, &tt, &l);
        fill(pos, l, e);
        pos++;
        k++;
      }
    }
  }
}

// TMA descriptors of a call, per tile shape: the stepped level's halo tile,
// the plain tile of the older level, the cc tile and (3D) the imaging
// accumulator tile.  2D uses shape 0 only.
struct Maps {
  CUtensorMap th[2], tp[2], tc[2], tg[2];
};

int make_tmaps(fwi_ctx* C, int B, int nslots, Maps* M) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return FWI_ERR_CUDA;
  const Layout& L = C->L;
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  auto encode = [&](CUtensorMap* m, int rank, void* base, const cuuint64_t* dims, const cuuint64_t* str,
                    const cuuint32_t* box) {
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, dims, str, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (L.ndim == 2) {
    const cuuint64_t dims[4] = {(cuuint64_t)L.SX, (cuuint64_t)L.NZ, (cuuint64_t)B, (cuuint64_t)nslots};
    const cuuint64_t str[3] = {(cuuint64_t)L.SX * 4, (cuuint64_t)L.SX * L.NZ * 4, (cuuint64_t)L.field * B * 4};
    const cuuint64_t cd[3] = {(cuuint64_t)L.SX, (cuuint64_t)L.NZ, (cuuint64_t)C->max_B};
    const cuuint64_t cs[2] = {(cuuint64_t)L.SX * 4, (cuuint64_t)L.field * 4};
    for (int sh = 0; sh < 2; sh++) {
      const cuuint32_t tz = (cuuint32_t)tile_rows2d(sh);
      const cuuint32_t bh[4] = {HX, tz + 2 * HALO, 1, 1}, bp[4] = {TX, tz, 1, 1}, cb[3] = {TX, tz, 1};
      if (!encode(&M->th[sh], 4, C->pool, dims, str, bh) || !encode(&M->tp[sh], 4, C->pool, dims, str, bp) ||
          !encode(&M->tc[sh], 3, C->c, cd, cs, cb))
        return FWI_ERR_CUDA;
      M->tg[sh] = M->tc[sh];  // unused by the 2D kernels
    }
    return FWI_OK;
  }
  const cuuint64_t dims[5] = {(cuuint64_t)L.SX, (cuuint64_t)L.NY, (cuuint64_t)L.NZ, (cuuint64_t)B,
                              (cuuint64_t)nslots};
  const cuuint64_t str[4] = {(cuuint64_t)L.SX * 4, (cuuint64_t)L.SX * L.NY * 4, (cuuint64_t)L.field * 4,
                             (cuuint64_t)L.field * B * 4};
  // cc per sample and the imaging accumulators (per wavefield or per pair), plain planes
  const cuuint64_t d4[4] = {(cuuint64_t)L.SX, (cuuint64_t)L.NY, (cuuint64_t)L.NZ, (cuuint64_t)C->max_B};
  const cuuint64_t s4[3] = {(cuuint64_t)L.SX * 4, (cuuint64_t)L.SX * L.NY * 4, (cuuint64_t)L.field * 4};
  for (int sh = 0; sh < 2; sh++) {
    const cuuint32_t ty = (cuuint32_t)tile_rows3(sh);
    const cuuint32_t bh[5] = {HX3, ty + 2 * HALO, 1, 1, 1}, bp[5] = {TX3, ty, 1, 1, 1}, b4[4] = {TX3, ty, 1, 1};
    if (!encode(&M->th[sh], 5, C->pool, dims, str, bh) || !encode(&M->tp[sh], 5, C->pool, dims, str, bp) ||
        !encode(&M->tc[sh], 4, C->c, d4, s4, b4) || !encode(&M->tg[sh], 4, C->G, d4, s4, b4))
      return FWI_ERR_CUDA;
  }
  return FWI_OK;
}

// Partition the pool into slots of B wavefields; re-zero it when the partition
// changes so that halos and the zero slot read as zero.
int partition_pool(fwi_ctx* C, int B, cudaStream_t st, long long* nslots) {
  const size_t slot_bytes = (size_t)C->L.field * B * 4;
  *nslots = (long long)(C->pool_bytes / slot_bytes);
  if (C->pool_B != B) {
    CK(cudaMemsetAsync(C->pool, 0, C->pool_bytes, st));
    C->pool_B = B;
  }
  return FWI_OK;
}

struct CallLists {  // byte offsets into the per-call list buffer; tile CSR lists per tile shape
  size_t inj_off[2], inj[2], smp_off[2], smp[2], shot_off, shot_id, shot_w, src_cnt, src_pos, src_amp, total;
};

// Per-call lists from the encoding: merged source points per wavefield (forward
// injection and adjoint sampling, tile CSR), shot lists for the residual, and
// source entries for the imaging term.
int build_call_lists(fwi_ctx* C, int nsamp, const int32_t* perm, const int8_t* w, const int32_t* sg, int nsg,
                     CallLists* cl, int* Emax_out, cudaStream_t st) {
  const int B = nsamp * nsg;
  std::vector<std::vector<Entry>> lists(B);
  std::vector<std::vector<std::pair<int, float>>> shots(B);
  int Emax = 0;
  for (int s = 0; s < nsamp; s++) {
    int o = 0;
    for (int j = 0; j < nsg; j++) {
      const int b = s * nsg + j;
      for (int k = 0; k < sg[j]; k++) {
        const int id = perm[(long long)s * C->ns + o + k];
        if (id < 0 || id >= C->ns) return FWI_ERR_ARG;
        const float wt = (float)w[(long long)s * C->ns + id];
        if (wt != 1.f && wt != -1.f) return FWI_ERR_ARG;
        shots[b].push_back({id, wt});
        const int z = C->src_zyx[3 * id], y = C->src_zyx[3 * id + 1], x = C->src_zyx[3 * id + 2];
        bool merged = false;
        for (auto& e : lists[b])
          if (e.z == z && e.y == y && e.x == x) {
            e.amp += wt;
            merged = true;
          }
        if (!merged) lists[b].push_back({z, y, x, 0, wt});
      }
      o += sg[j];
      for (size_t e = 0; e < lists[b].size(); e++) lists[b][e].col = (int)e;
      Emax = std::max(Emax, (int)lists[b].size());
    }
  }
  if (Emax > C->Emax) return FWI_ERR_ARG;
  int nent = 0;
  for (auto& l : lists) nent += (int)l.size();
  int nshot = 0;
  for (auto& l : shots) nshot += (int)l.size();
  size_t p = 0;
  auto take = [&](size_t bytes) {
    size_t r = p;
    p = (p + bytes + 255) / 256 * 256;
    return r;
  };
  const int nsh = 2;  // both tile shapes (3D: 64 x 16 and pairs; 2D: 128 x 32 and 128 x 24)
  for (int sh = 0; sh < 2; sh++) {
    const int sh_eff = sh < nsh ? sh : 0;  // 2D: shape 1 aliases shape 0
    if (sh != sh_eff) {
      cl->inj_off[sh] = cl->inj_off[0];
      cl->inj[sh] = cl->inj[0];
      cl->smp_off[sh] = cl->smp_off[0];
      cl->smp[sh] = cl->smp[0];
      continue;
    }
    cl->inj_off[sh] = take((size_t)B * (C->ntiles_s[sh] + 1) * 4);
    cl->inj[sh] = take((size_t)std::max(nent, 1) * 16);
    cl->smp_off[sh] = take((size_t)B * (C->ntiles_s[sh] + 1) * 4);
    cl->smp[sh] = take((size_t)std::max(nent, 1) * 16);
  }
  cl->shot_off = take((size_t)(B + 1) * 4);
  cl->shot_id = take((size_t)std::max(nshot, 1) * 4);
  cl->shot_w = take((size_t)std::max(nshot, 1) * 4);
  cl->src_cnt = take((size_t)B * 4);
  cl->src_pos = take((size_t)B * std::max(C->Emax, 1) * 8);
  cl->src_amp = take((size_t)B * std::max(C->Emax, 1) * 4);
  cl->total = p;
  if (p > C->list_bytes) return FWI_ERR_ARG;
  // this turn's staging buffer: its previous upload (kStaging uploads ago)
  // must have left it
  const int turn = C->list_turn;
  C->list_turn = (turn + 1) % kStaging;
  CK(cudaEventSynchronize(C->ev_list[turn]));
  unsigned char* h = C->hlist[turn];
  const float inv_vol = (float)(1.0 / C->cell_volume);
  const bool is3d = C->L.ndim == 3;
  for (int sh = 0; sh < nsh; sh++) {
    build_csr(C, lists, sh, reinterpret_cast<int*>(h + cl->inj_off[sh]), [&](int pos, int local, const Entry& e) {
      int4 v;
      v.x = local;
      v.y = 0;
      float a = e.amp * inv_vol;
      memcpy(&v.z, &a, 4);
      v.w = e.z;
      reinterpret_cast<int4*>(h + cl->inj[sh])[pos] = v;
    });
    build_csr(C, lists, sh, reinterpret_cast<int*>(h + cl->smp_off[sh]), [&](int pos, int local, const Entry& e) {
      if (is3d)
        reinterpret_cast<int4*>(h + cl->smp[sh])[pos] = make_int4(local, e.col, e.z, 0);
      else
        reinterpret_cast<int2*>(h + cl->smp[sh])[pos] = make_int2(local, e.col);
    });
  }
  int* so = reinterpret_cast<int*>(h + cl->shot_off);
  int* sid = reinterpret_cast<int*>(h + cl->shot_id);
  float* sw = reinterpret_cast<float*>(h + cl->shot_w);
  int q = 0;
  for (int b = 0; b < B; b++) {
    so[b] = q;
    for (auto& pr : shots[b]) {
      sid[q] = pr.first;
      sw[q] = pr.second;
      q++;
    }
  }
  so[B] = q;
  int* cnt = reinterpret_cast<int*>(h + cl->src_cnt);
  long long* pos = reinterpret_cast<long long*>(h + cl->src_pos);
  float* amp = reinterpret_cast<float*>(h + cl->src_amp);
  for (int b = 0; b < B; b++) {
    cnt[b] = (int)lists[b].size();
    for (size_t e = 0; e < lists[b].size(); e++) {
      const Entry& en = lists[b][e];
      pos[(size_t)b * C->Emax + e] = C->L.off(en.z, en.y, en.x);
      amp[(size_t)b * C->Emax + e] = en.amp * inv_vol;
    }
  }
  CK(cudaMemcpyAsync(C->dlist, h, cl->total, cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(C->ev_list[turn], st));
  *Emax_out = Emax;
  return FWI_OK;
}

int validate_call(fwi_ctx* C, const float* vel, int nsamp, const int32_t* perm, const int8_t* w, const int32_t* sg,
                  int nsg) {
  if (!C || !vel || !perm || !w || !sg || nsamp < 1 || nsg < 1) return FWI_ERR_ARG;
  if ((long long)nsamp * nsg > C->max_B) return FWI_ERR_ARG;
  long long tot = 0;
  for (int j = 0; j < nsg; j++) {
    if (sg[j] < 1) return FWI_ERR_ARG;
    tot += sg[j];
  }
  if (tot > C->ns) return FWI_ERR_ARG;
  return FWI_OK;
}

// 3D tile shape of the forward kernel (the autotuned variant's bit 2) and of
// the adjoint kernel: 64 x 16 tiles unless a forced variant sets bit 2 (pair
// tiles, for a sample with an even number of supergathers).  The autotuner
// does not choose the adjoint's shape, since the pair form sums the imaging
// term in another order and a timing-dependent choice would make results
// depend on the run.  2D: variant bit 1 (128 x 32 or 128 x 24 tiles, the same
// arithmetic per point), for the forward and the adjoint alike.
int shape_fwd(const fwi_ctx* C) {
  if (C->var[0] < 0) return 0;
  return C->L.ndim == 3 ? (C->var[0] >> 2) & 1 : (C->var[0] >> 1) & 1;
}
int shape_adj(const fwi_ctx* C, int nsg) {
  if (C->L.ndim == 2) return C->var[1] >= 0 ? (C->var[1] >> 1) & 1 : 0;
  return nsg % 2 == 0 && C->var[1] >= 0 && (C->var[1] & 4) ? 1 : 0;
}

StepParams base_params(fwi_ctx* C, int B, int nsg, int sh = 0) {
  StepParams P;
  memset(&P, 0, sizeof(P));
  P.pool = C->pool;
  P.slot_elems = C->L.field * B;
  P.c = C->c;
  P.gtab = C->gtab;
  P.grad = C->G;
  P.smp_off = C->zero_off;  // "no sampling points" unless a call sets a list
  P.smp_bstride = 0;
  P.nsg = nsg;
  P.ntx = C->ntx;
  P.ntiles = C->ntiles_s[sh];
  P.pair3 = sh;
  P.status = C->status;
  return P;
}

// Steps descs[off, off + n) of the current call: one multi-step launch in 2D
// and for the persistent 3D variants (progress flags zeroed first), else one
// launch per step.  P carries its tile shape (P.pair3) and that shape's lists.
int run_steps(fwi_ctx* C, bool adj, StepParams P, int off, int n, int nsamp, int B, const Maps& M, cudaStream_t st,
              long long* launches) {
  if (n <= 0) return FWI_OK;
  const int sh = P.pair3;
  if (C->L.ndim == 3) {
    const int v = C->var[adj ? 1 : 0];
    P.order3 = v & 1;
    P.zpair3 = (v >> 1) & 1;
    P.ctas_per_sm3 = (v >> 3) & 1;
    if (multi_step3(v)) {
      const int units = sh ? B / 2 : B;
      P.steps = C->desc + off;
      P.nsteps = n;
      P.done = C->done;
      CK(cudaMemsetAsync(C->done, 0, (size_t)units * P.ntiles * 4, st));
      CK(launch_step3d(adj, M.th[sh], M.tp[sh], M.tc[sh], M.tg[sh], C->L, C->K, P, B, st));
      *launches += 1;
      return FWI_OK;
    }
    P.steps = nullptr;
    for (int i = 0; i < n; i++) {
      const StepDesc& d = C->descs[off + i];
      P.s_cur = d.cur;
      P.s_prev = d.prev;
      P.s_out = d.out;
      P.s_snap = d.snap;
      P.t = d.t;
      CK(launch_step3d(adj, M.th[sh], M.tp[sh], M.tc[sh], M.tg[sh], C->L, C->K, P, B, st));
    }
    *launches += n;
    return FWI_OK;
  }
  P.steps = C->desc + off;
  P.nsteps = n;
  P.done = C->done;
  CK(cudaMemsetAsync(C->done, 0, (size_t)nsamp * P.ntiles * 4, st));
  CK(launch_step2d(adj, C->var[adj ? 1 : 0], M.th[sh], M.tp[sh], M.tc[sh], C->L, C->K, P, nsamp, st));
  *launches += 1;
  return FWI_OK;
}

// Copies the call's step descriptors (C->descs) to the device.
int upload_descs(fwi_ctx* C, cudaStream_t st) {
  const size_t n = C->descs.size();
  if (n > C->desc_cap) return FWI_ERR_ARG;
  const int turn = C->desc_turn;  // staging buffer of this upload (see kStaging)
  C->desc_turn = (turn + 1) % kStaging;
  CK(cudaEventSynchronize(C->ev_desc[turn]));
  memcpy(C->hdesc[turn], C->descs.data(), n * sizeof(StepDesc));
  CK(cudaMemcpyAsync(C->desc, C->hdesc[turn], n * sizeof(StepDesc), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(C->ev_desc[turn], st));
  return FWI_OK;
}

StepDesc make_desc(int cur, int prev, int out, int snap, int t) {
  StepDesc d;
  d.cur = cur;
  d.prev = prev;
  d.out = out;
  d.snap = snap;
  d.t = t;
  d.pad[0] = d.pad[1] = d.pad[2] = 0;
  return d;
}

// Step-kernel variants: 2D ring depths (stencil.cu).  3D variant v: bit 0
// the CTA order (tile-major, wavefield-fastest), bit 1 two z levels per march
// step, bit 2 the tile shape (64 x 16, or 64 x 8 pair tiles when a sample
// has an even number of supergathers; for the adjoint only when forced, see
// shape_adj), bit 3 a persistent grid of one CTA per SM running its columns
// back to back (else one CTA per column), bit 4 (with bit 3) all steps of a
// phase in one cooperative launch, chained column by column by progress
// flags (else one launch per step).  Bit 4 without bit 3 is not a variant.
int num_variants(const fwi_ctx* C, bool adj) { return C->L.ndim == 3 ? kMaxVariants : num_variants2d(adj); }
const char* variant_name(const fwi_ctx* C, bool adj, int v) {
  if (C->L.ndim == 2) return variant2d_name(adj, v);
  static char names[2][kMaxVariants][96];
  static bool init = false;
  if (!init) {
    for (int a = 0; a < 2; a++)
      for (int i = 0; i < kMaxVariants; i++)
        snprintf(names[a][i], sizeof(names[a][i]), "%s %s %s, %d level%s%s%s", a ? "adj3d" : "fwd3d",
                 (i & 4) ? "64x8 pairs" : "64x16", (i & 1) ? "wavefield-fastest" : "tile-major", (i & 2) ? 2 : 1,
                 (i & 2) ? "s" : "", (i & 8) ? ", persistent" : "", multi_step3(i) ? " multi-step" : "");
    init = true;
  }
  if (v < 0 || v >= kMaxVariants || ((v & 16) && !(v & 8))) return "-";
  if (adj && C->adj_pair != ((v >> 2) & 1)) return names[1][v ^ 4];  // the shape the adjoint ran on
  return names[adj ? 1 : 0][v];
}

// kTuneSteps steps of variant v: one multi-step launch in 2D and for the
// persistent 3D variants (step table P.steps), else one launch per step
// (slots from td).  P carries the variant's tile shape and lists.
cudaError_t launch_tune(fwi_ctx* C, bool adj, int v, StepParams P, const StepDesc* td, int nsamp, int B,
                        const Maps& M, cudaStream_t st) {
  if (C->L.ndim == 3) {
    P.order3 = v & 1;
    P.zpair3 = (v >> 1) & 1;
    P.ctas_per_sm3 = (v >> 3) & 1;
    const int sh = P.pair3;
    if (multi_step3(v)) {
      cudaError_t e = cudaMemsetAsync(C->done, 0, (size_t)(sh ? B / 2 : B) * P.ntiles * 4, st);
      if (e != cudaSuccess) return e;
      return launch_step3d(adj, M.th[sh], M.tp[sh], M.tc[sh], M.tg[sh], C->L, C->K, P, B, st);
    }
    P.steps = nullptr;
    for (int i = 0; i < kTuneSteps; i++) {
      P.s_cur = td[i].cur;
      P.s_prev = td[i].prev;
      P.s_out = td[i].out;
      P.s_snap = td[i].snap;
      cudaError_t e = launch_step3d(adj, M.th[sh], M.tp[sh], M.tc[sh], M.tg[sh], C->L, C->K, P, B, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaMemsetAsync(C->done, 0, (size_t)nsamp * P.ntiles * 4, st);
  if (e != cudaSuccess) return e;
  return launch_step2d(adj, v, M.th[P.pair3], M.tp[P.pair3], M.tc[P.pair3], C->L, C->K, P, nsamp, st);
}

// Autotuner: time every variant of the forward and adjoint step kernels on
// this call's shape (B wavefields over the real tiles, whatever the three ring
// slots hold, no injection or sampling) and keep the fastest.  Runs once per
// wavefield count; synchronises the stream while it times.  All variants give
// bit-identical results.  The 3D adjoint variant writes the imaging
// accumulators, which every gradient chunk clears after tuning.
int autotune(fwi_ctx* C, int nsamp, int nsg, const Maps& M, long long nslots, cudaStream_t st) {
  const int B = nsamp * nsg;
  if (C->tuned_B == B && C->tuned_nsg == nsg && C->var[0] >= 0 && C->var[1] >= 0) {
    C->adj_pair = shape_adj(C, nsg);
    return FWI_OK;
  }
  C->var[1] = C->forced[1] >= 0 ? C->forced[1] : -1;
  C->adj_pair = shape_adj(C, nsg);
  // timing steps with the traffic of real ones: the three ring slots rotate
  // (whatever they hold), the snapshot comes from a fourth slot when there is one
  StepDesc td[kTuneSteps];
  for (int i = 0; i < kTuneSteps; i++)
    td[i] = make_desc(Plan::RING + i % 3, Plan::RING + (i + 2) % 3, Plan::RING + (i + 1) % 3,
                      nslots > Plan::QR ? Plan::QR : Plan::ZERO, 0);
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(C->tdesc, td, sizeof(td), cudaMemcpyHostToDevice));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int adj = 0; adj < 2; adj++) {
    const int nv = num_variants(C, adj != 0);
    for (int v = 0; v < kMaxVariants; v++) C->tune_ms[adj][v] = -1.f;
    if (C->forced[adj] >= 0 && C->forced[adj] < nv) {
      // a forced 3D pair-tile forward needs an even number of supergathers:
      // otherwise the same variant with 64 x 16 tiles
      C->var[adj] = (C->L.ndim == 3 && !adj && nsg % 2) ? (C->forced[adj] & ~4) : C->forced[adj];
      continue;
    }
    int best = -1;
    float best_ms = 1e30f;
    for (int v = 0; v < nv && v < kMaxVariants; v++) {
      if (C->L.ndim == 3 && adj && (v & 4)) continue;  // the adjoint's tile shape is not tuned (shape_adj)
      if (C->L.ndim == 3 && (v & 16) && !(v & 8)) continue;  // multi-step needs the persistent grid
      // pair tiles need an even number of supergathers per sample
      const int sh = C->L.ndim == 3 ? (adj ? shape_adj(C, nsg) : (v >> 2) & 1) : (v >> 1) & 1;
      if (C->L.ndim == 3 && sh && nsg % 2) continue;
      StepParams P = base_params(C, B, nsg, sh);
      P.inj_off = C->zero_off;
      P.inj_bstride = 0;
      P.inj = C->rec_inj[sh];
      P.series = C->wav;
      P.steps = C->tdesc;
      P.nsteps = kTuneSteps;
      P.done = C->done;
      if (launch_tune(C, adj != 0, v, P, td, nsamp, B, M, st) != cudaSuccess) {
        cudaGetLastError();  // variant does not fit this device: skip it
        continue;
      }
      CK(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; r++) CK(launch_tune(C, adj != 0, v, P, td, nsamp, B, M, st));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      C->tune_ms[adj][v] = ms / (3.f * kTuneSteps);  // per step
      if (ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    if (best < 0) return FWI_ERR_CUDA;
    C->var[adj] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  C->tuned_B = B;
  C->tuned_nsg = nsg;
  return FWI_OK;
}

void prof_mark(fwi_ctx* C, int i, cudaStream_t st) {
  if (C->prof) cudaEventRecord(C->ev[i], st);
}

}  // namespace

// ------------------------------------------------------------- public ABI --

extern "C" {

const char* fwi_status_string(int s) {
  switch (s) {
    case FWI_OK: return "ok";
    case FWI_ERR_ARG: return "invalid argument";
    case FWI_ERR_CFL: return "stability (CFL) bound violated";
    case FWI_ERR_OOM: return "out of memory";
    case FWI_ERR_CUDA: return "CUDA error";
    case FWI_ERR_NONFINITE: return "non-finite misfit";
    case FWI_ERR_TIMEOUT: return "device wait timed out";
    case FWI_ERR_BOUNDS: return "device index check failed";
    default: return "unknown status";
  }
}

const char* fwi_last_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "no error" : cudaGetErrorString(g_last_cuda_error);
}

int fwi_encode(uint64_t seed, uint64_t iter, int ns, int32_t* perm, int8_t* w) {
  if (ns < 1 || !perm || !w) return FWI_ERR_ARG;
  const uint64_t G = 0x9e3779b97f4a7c15ULL;
  const uint64_t key = mix64(seed ^ mix64(iter));
  for (int i = 0; i < ns; i++) w[i] = (mix64(key + (uint64_t)(i + 1) * G) >> 63) ? -1 : 1;
  for (int i = 0; i < ns; i++) perm[i] = i;
  for (int i = ns - 1; i >= 1; i--) {
    const uint64_t u = mix64(key + ((uint64_t)ns + (uint64_t)(ns - 1 - i) + 1) * G);
    const uint64_t j = (uint64_t)(((unsigned __int128)u * (unsigned __int128)(i + 1)) >> 64);
    std::swap(perm[i], perm[j]);
  }
  return FWI_OK;
}

int fwi_create(const fwi_grid* g, const fwi_geom* geom, int max_wavefields, size_t budget, fwi_ctx** out) {
  if (!out) return FWI_ERR_ARG;
  *out = nullptr;
  int rc = check_grid(g);
  if (rc != FWI_OK) return rc;
  if (!geom || geom->ns < 1 || geom->nr < 1 || !geom->src || !geom->rec || max_wavefields < 1) return FWI_ERR_ARG;
  fwi_ctx* C = new (std::nothrow) fwi_ctx();
  if (!C) return FWI_ERR_OOM;
  C->g = *g;
  C->L = make_layout(g);
  C->K = make_coef(g);
  C->ns = geom->ns;
  C->nr = geom->nr;
  C->max_B = max_wavefields;
  C->cell_volume = g->hz * g->hx * (g->ndim == 3 ? g->hy : 1.0);
  C->vmax_cfl = g->sponge_vmax;
  const Layout& L = C->L;
  auto conv = [&](const int32_t* p, int n, std::vector<int>& dst) {
    for (int i = 0; i < n; i++) {
      const int iz = p[3 * i], iy = g->ndim == 3 ? p[3 * i + 1] : 0, ix = p[3 * i + 2];
      if (iz < 0 || iz >= L.nz || iy < 0 || iy >= L.ny || ix < 0 || ix >= L.nx) return false;
      dst.push_back(iz + L.nb);
      dst.push_back(g->ndim == 3 ? iy + L.nb : 0);
      dst.push_back(ix + L.nb);
    }
    return true;
  };
  if (!conv(geom->src, geom->ns, C->src_zyx) || !conv(geom->rec, geom->nr, C->rec_zyx)) {
    delete C;
    return FWI_ERR_ARG;
  }
  for (int a = 0; a < C->nr; a++)
    for (int b = a + 1; b < C->nr; b++)
      if (C->rec_zyx[3 * a] == C->rec_zyx[3 * b] && C->rec_zyx[3 * a + 1] == C->rec_zyx[3 * b + 1] &&
          C->rec_zyx[3 * a + 2] == C->rec_zyx[3 * b + 2]) {
        delete C;
        return FWI_ERR_ARG;
      }
  C->ntx = g->ndim == 3 ? (L.nxp + TX3 - 1) / TX3 : (L.nxp + TX - 1) / TX;
  C->ntz = (L.nzp + TZ - 1) / TZ;
  C->nty = (L.nyp + TY3 - 1) / TY3;
  C->ntiles = C->ntx * (g->ndim == 3 ? C->nty : C->ntz);
  C->ntiles_s[0] = C->ntiles;
  C->ntiles_s[1] = g->ndim == 3 ? C->ntx * ((L.nyp + tile_rows3(1) - 1) / tile_rows3(1))
                                 : C->ntx * ((L.nzp + tile_rows2d(1) - 1) / tile_rows2d(1));
  C->Emax = std::min(C->ns, 4096);
  C->nblk = 64;

  const int B = max_wavefields;
  const size_t fbytes = (size_t)L.field * 4;
  rc = FWI_ERR_OOM;
  auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max(bytes, (size_t)256)) == cudaSuccess; };
  if (!alloc((void**)&C->c, fbytes * B) || !alloc((void**)&C->G, fbytes * B) ||
      !alloc((void**)&C->wav, (size_t)g->nt * 4) || !alloc((void**)&C->dpred, (size_t)B * g->nt * C->nr * 4) ||
      !alloc((void**)&C->part, (size_t)B * C->nblk * 8) ||
      !alloc((void**)&C->qsrc, (size_t)B * g->nt * C->Emax * 4) ||
      !alloc((void**)&C->stmp, (size_t)B * C->Emax * 4) || !alloc((void**)&C->status, 64)) {
    fwi_destroy(C);
    return FWI_ERR_OOM;
  }
  // receiver lists, shared by every wavefield, per tile shape
  for (int sh = 0; sh < 2; sh++) {
    std::vector<std::vector<Entry>> rl(1);
    for (int r = 0; r < C->nr; r++) rl[0].push_back({C->rec_zyx[3 * r], C->rec_zyx[3 * r + 1], C->rec_zyx[3 * r + 2], r, 1.f});
    std::vector<int> off(C->ntiles_s[sh] + 1);
    std::vector<int2> smp(C->nr);
    std::vector<int4> smp4(C->nr);
    std::vector<int4> inj(C->nr);
    build_csr(C, rl, sh, off.data(), [&](int pos, int local, const Entry& e) {
      smp[pos] = make_int2(local, e.col);
      smp4[pos] = make_int4(local, e.col, e.z, 0);
      int4 v;
      v.x = local;
      v.y = e.col;
      float one = 1.f;
      memcpy(&v.z, &one, 4);
      v.w = e.z;
      inj[pos] = v;
    });
    if (!alloc((void**)&C->rec_off[sh], off.size() * 4) || (g->ndim == 2 && !alloc((void**)&C->rec_smp[sh], smp.size() * 8)) ||
        !alloc((void**)&C->rec_smp4[sh], smp4.size() * 16) || !alloc((void**)&C->rec_inj[sh], inj.size() * 16)) {
      fwi_destroy(C);
      return FWI_ERR_OOM;
    }
    if (cudaMemcpy(C->rec_off[sh], off.data(), off.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        (g->ndim == 2 && cudaMemcpy(C->rec_smp[sh], smp.data(), smp.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) ||
        cudaMemcpy(C->rec_smp4[sh], smp4.data(), smp4.size() * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(C->rec_inj[sh], inj.data(), inj.size() * 16, cudaMemcpyHostToDevice) != cudaSuccess) {
      fwi_destroy(C);
      return FWI_ERR_CUDA;
    }
  }
  const int ntiles_max = std::max(C->ntiles_s[0], C->ntiles_s[1]);
  if (!alloc((void**)&C->zero_off, (size_t)(ntiles_max + 1) * 4) ||
      cudaMemset(C->zero_off, 0, (size_t)(ntiles_max + 1) * 4) != cudaSuccess) {
    fwi_destroy(C);
    return FWI_ERR_OOM;
  }
  {  // per-axis gamma*dt of the sponge
    double hmin = std::min(g->hz, g->hx);
    if (g->ndim == 3) hmin = std::min(hmin, g->hy);
    const double gmax = g->nb > 0 ? 3.0 * g->sponge_vmax * log(1.0 / g->sponge_R) / (2.0 * g->nb * hmin) : 0.0;
    std::vector<float> t;
    auto axis = [&](int n, int np) {
      for (int i = 0; i < np; i++) {
        const int d = i < g->nb ? g->nb - i : (i >= g->nb + n ? i - (g->nb + n - 1) : 0);
        const double f = g->nb > 0 ? (double)d / g->nb : 0.0;
        t.push_back((float)(gmax * g->dt * f * f));
      }
    };
    axis(g->nz, L.nzp);
    if (g->ndim == 3) axis(g->ny, L.nyp); else t.push_back(0.f);
    axis(g->nx, L.nxp);
    if (!alloc((void**)&C->gtab, t.size() * 4) ||
        cudaMemcpy(C->gtab, t.data(), t.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
      fwi_destroy(C);
      return FWI_ERR_OOM;
    }
  }
  // per-call list buffers (worst case: every shot its own node)
  // (3D: the tile CSR lists of both tile shapes)
  C->list_bytes = (size_t)B * (C->ntiles_s[0] + C->ntiles_s[1] + 2) * 8 + (size_t)B * C->Emax * (2 * 32 + 8 + 4) +
                  (size_t)(B + 1) * 4 + (size_t)B * C->ns * 8 + (size_t)B * 4 + 64 * 256;
  if (!alloc((void**)&C->dlist, C->list_bytes) ||
      [&] {
        for (int i = 0; i < kStaging; i++)
          if (cudaHostAlloc((void**)&C->hlist[i], C->list_bytes, cudaHostAllocDefault) != cudaSuccess) return true;
        return false;
      }()) {
    fwi_destroy(C);
    return FWI_ERR_OOM;
  }
  if ([&] {
        for (int i = 0; i < kStaging; i++)
          if (cudaEventCreateWithFlags(&C->ev_list[i], cudaEventDisableTiming) != cudaSuccess ||
              cudaEventCreateWithFlags(&C->ev_desc[i], cudaEventDisableTiming) != cudaSuccess)
            return true;
        return false;
      }()) {
    fwi_destroy(C);
    return FWI_ERR_CUDA;
  }
  // step descriptors: forward, recomputed and adjoint steps of one call
  C->desc_cap = 3 * (size_t)g->nt + 16;
  if (!alloc((void**)&C->desc, C->desc_cap * sizeof(StepDesc)) ||
      [&] {
        for (int i = 0; i < kStaging; i++)
          if (cudaHostAlloc((void**)&C->hdesc[i], C->desc_cap * sizeof(StepDesc), cudaHostAllocDefault) !=
              cudaSuccess)
            return true;
        return false;
      }() ||
      !alloc((void**)&C->tdesc, kTuneSteps * sizeof(StepDesc)) ||
      !alloc((void**)&C->done, (size_t)B * std::max(C->ntiles_s[0], C->ntiles_s[1]) * 4)) {
    fwi_destroy(C);
    return FWI_ERR_OOM;
  }

  for (int i = 0; i < 5; i++)
    if (cudaEventCreate(&C->ev[i]) != cudaSuccess) {
      fwi_destroy(C);
      return FWI_ERR_CUDA;
    }
  // wavefield pool
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  size_t want = budget ? budget : (size_t)(0.8 * (double)fr);
  const size_t min_pool = fbytes * B * 4;
  if (want < min_pool || want > fr) {
    fwi_destroy(C);
    return FWI_ERR_OOM;
  }
  C->pool_bytes = want / 256 * 256;
  if (!alloc((void**)&C->pool, C->pool_bytes)) {
    fwi_destroy(C);
    return FWI_ERR_OOM;
  }
  if (cudaMemset(C->status, 0, 64) != cudaSuccess || cudaMemset(C->c, 0, fbytes * B) != cudaSuccess ||
      launch_wavelet(g->nt, g->dt, g->f0, g->t0, C->wav, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    fwi_destroy(C);
    return FWI_ERR_CUDA;
  }
  *out = C;
  return FWI_OK;
}

void fwi_destroy(fwi_ctx* C) {
  if (!C) return;
  cudaFree(C->pool);
  cudaFree(C->c);
  cudaFree(C->G);
  cudaFree(C->wav);
  cudaFree(C->dpred);
  cudaFree(C->part);
  cudaFree(C->qsrc);
  cudaFree(C->stmp);
  cudaFree(C->status);
  for (int sh = 0; sh < 2; sh++) {
    cudaFree(C->rec_off[sh]);
    cudaFree(C->rec_smp4[sh]);
    cudaFree(C->rec_inj[sh]);
  }
  cudaFree(C->rec_smp[0]);
  cudaFree(C->rec_smp[1]);
  cudaFree(C->dlist);
  cudaFree(C->zero_off);
  cudaFree(C->gtab);
  cudaFree(C->desc);
  cudaFree(C->tdesc);
  cudaFree(C->done);
  for (int i = 0; i < kStaging; i++) {
    if (C->hlist[i]) cudaFreeHost(C->hlist[i]);
    if (C->hdesc[i]) cudaFreeHost(C->hdesc[i]);
    if (C->ev_list[i]) cudaEventDestroy(C->ev_list[i]);
    if (C->ev_desc[i]) cudaEventDestroy(C->ev_desc[i]);
  }
  for (int i = 0; i < 5; i++)
    if (C->ev[i]) cudaEventDestroy(C->ev[i]);
  delete C;
}

// Forward steps 0..nt-1 of fwi_forward on a three-slot ring (no snapshots kept).
static void append_forward_descs(fwi_ctx* C) {
  for (int n = 0; n < C->g.nt; n++)
    C->descs.push_back(make_desc(n <= 0 ? 0 : 1 + n % 3, n - 1 <= 0 ? 0 : 1 + (n - 1) % 3, 1 + (n + 1) % 3,
                                 Plan::ZERO, n));
}

// Step descriptors of one gradient chunk in launch order: the first forward
// pass (steps 0..nt-1), then per segment j from the last, its recomputed
// forward steps and its adjoint steps; rc_* / ad_* give each segment's two
// phases as (offset, count) into descs.
static void gradient_descs(const Plan& plan, int nt, std::vector<StepDesc>& descs, std::vector<int>& rc_off,
                           std::vector<int>& rc_n, std::vector<int>& ad_off, std::vector<int>& ad_n) {
  descs.clear();
  for (int n = 0; n < nt; n++)
    descs.push_back(make_desc(plan.fslot(n), plan.fslot(n - 1), plan.fslot(n + 1), Plan::ZERO, n));
  rc_off.assign(plan.jL + 1, 0);
  rc_n.assign(plan.jL + 1, 0);
  ad_off.assign(plan.jL + 1, 0);
  ad_n.assign(plan.jL + 1, 0);
  for (int j = plan.jL; j >= 0; j--) {
    const int m0 = j * plan.K, m1 = std::min((j + 1) * plan.K, nt);  // snapshots m0..m1-1
    rc_off[j] = (int)descs.size();
    if (j < plan.jL)
      for (int n = m0; n <= m1 - 2; n++)
        descs.push_back(make_desc(plan.rslot(j, n), plan.rslot(j, n - 1), plan.rslot(j, n + 1), Plan::ZERO, n));
    rc_n[j] = (int)descs.size() - rc_off[j];
    ad_off[j] = (int)descs.size();
    for (int k = m1; k >= m0 + 1; k--)
      descs.push_back(make_desc(plan.qslot(k + 1), plan.qslot(k + 2), plan.qslot(k), plan.snap(j, k - 1), k - 1));
    ad_n[j] = (int)descs.size() - ad_off[j];
  }
}

static int run_forward_loop(fwi_ctx* C, int nsamp, int nsg, const CallLists& cl, const Maps& M, int desc_off,
                            float* dout, cudaStream_t st) {
  const int B = nsamp * nsg;
  const int sh = shape_fwd(C);
  StepParams P = base_params(C, B, nsg, sh);
  P.inj_off = reinterpret_cast<const int*>(C->dlist + cl.inj_off[sh]);
  P.inj_bstride = C->ntiles_s[sh] + 1;
  P.inj = reinterpret_cast<const int4*>(C->dlist + cl.inj[sh]);
  P.series = C->wav;
  P.series_bstride = 0;
  P.series_ld = 1;
  P.smp_off = C->rec_off[sh];
  P.smp_bstride = 0;
  if (C->L.ndim == 3)
    P.smp4 = C->rec_smp4[sh];
  else
    P.smp = C->rec_smp[sh];
  P.smp_out = dout;
  P.smp_bstride_out = (long long)C->g.nt * C->nr;
  P.smp_ld = C->nr;
  return run_steps(C, false, P, desc_off, C->g.nt, nsamp, B, M, st, &C->launches[0]);
}

int fwi_forward(fwi_ctx* C, const float* vel, int nsamp, const int32_t* perm, const int8_t* w, const int32_t* sg,
                int nsg, float* d_pred, void* stream) {
  int rc = validate_call(C, vel, nsamp, perm, w, sg, nsg);
  if (rc != FWI_OK) return rc;
  if (!d_pred) return FWI_ERR_ARG;
  Ranges nv("fwi_forward");
  cudaStream_t st = (cudaStream_t)stream;
  const int B = nsamp * nsg;
  long long nslots;
  if ((rc = partition_pool(C, B, st, &nslots)) != FWI_OK) return rc;
  if (nslots < 4) return FWI_ERR_OOM;
  Maps M;
  if ((rc = make_tmaps(C, B, (int)nslots, &M)) != FWI_OK) return rc;
  if ((rc = autotune(C, nsamp, nsg, M, nslots, st)) != FWI_OK) return rc;
  CallLists cl;
  int Emax;
  if ((rc = build_call_lists(C, nsamp, perm, w, sg, nsg, &cl, &Emax, st)) != FWI_OK) return rc;
  for (int i = 0; i < 4; i++) C->launches[i] = 0;
  C->last_was_gradient = false;
  prof_mark(C, 0, st);
  C->descs.clear();
  append_forward_descs(C);
  if ((rc = upload_descs(C, st)) != FWI_OK) return rc;
  CK(launch_expand(C->L, vel, nsamp, C->g.dt, C->gtab, C->c, (float)C->vmax_cfl, C->status, st));
  if ((rc = run_forward_loop(C, nsamp, nsg, cl, M, 0, d_pred, st)) != FWI_OK) return rc;
  prof_mark(C, 1, st);
  prof_mark(C, 2, st);
  prof_mark(C, 3, st);
  prof_mark(C, 4, st);
  return FWI_OK;
}

// One chunk of samples through forward, residual/misfit, reverse sweep and
// fold.  The pool is partitioned for Bpart >= nsamp*nsg wavefields, so every
// chunk of a call (the last one may be smaller) shares one slot layout.
// With cot != nullptr the chunk applies the transposed Jacobian of the
// records instead: cot (this chunk's [B][nt][nr] cotangent) takes the place
// of the residual and no misfit is formed.
static int gradient_chunk(fwi_ctx* C, const float* vel, int nsamp, const int32_t* perm, const int8_t* w,
                          const int32_t* sg, int nsg, const float* d_obs, const float* cot, double sigma_y,
                          double scale, float* grad, double* misfit, cudaStream_t st, int Bpart) {
  int rc;
  const int B = nsamp * nsg;
  const int nt = C->g.nt, nr = C->nr;
  long long nslots;
  if ((rc = partition_pool(C, Bpart, st, &nslots)) != FWI_OK) return rc;
  Plan plan;
  if (!make_plan(nt, nslots, &plan)) return FWI_ERR_OOM;
  C->plan = plan;
  C->slots_avail = nslots;
  Maps M;
  if ((rc = make_tmaps(C, Bpart, (int)nslots, &M)) != FWI_OK) return rc;
  if ((rc = autotune(C, Bpart / nsg, nsg, M, nslots, st)) != FWI_OK) return rc;
  CallLists cl;
  int Emax;
  if ((rc = build_call_lists(C, nsamp, perm, w, sg, nsg, &cl, &Emax, st)) != FWI_OK) return rc;

  Ranges nv("gradient chunk");
  nv.phase("forward");
  prof_mark(C, 0, st);
  std::vector<int> rc_off, rc_n, ad_off, ad_n;
  gradient_descs(plan, nt, C->descs, rc_off, rc_n, ad_off, ad_n);
  if ((rc = upload_descs(C, st)) != FWI_OK) return rc;

  CK(launch_expand(C->L, vel, nsamp, C->g.dt, C->gtab, C->c, (float)C->vmax_cfl, C->status, st));
  C->launches[0] += 1;
  // imaging accumulators: one per sample (2D), per pair of supergathers (3D
  // pair tiles) or per wavefield (3D)
  const int sh_a = shape_adj(C, nsg);
  const int wf_per_acc = C->L.ndim == 2 ? nsg : (sh_a ? 2 : 1);
  CK(cudaMemsetAsync(C->G, 0, (size_t)C->L.field * (B / wf_per_acc) * 4, st));
  if ((rc = run_forward_loop(C, nsamp, nsg, cl, M, 0, C->dpred, st)) != FWI_OK) return rc;
  prof_mark(C, 1, st);

  nv.phase(cot ? "cotangent" : "residual and misfit");
  if (cot) {  // the given cotangent is the adjoint source
    CK(cudaMemcpyAsync(C->dpred, cot, (size_t)B * nt * nr * 4, cudaMemcpyDeviceToDevice, st));
  } else {  // residual (rhat overwrites dpred) and misfit
    const double inv_s2 = 1.0 / (sigma_y * sigma_y);
    CK(launch_residual(B, nt, nr, C->dpred, d_obs, reinterpret_cast<const int*>(C->dlist + cl.shot_off),
                       reinterpret_cast<const int*>(C->dlist + cl.shot_id),
                       reinterpret_cast<const float*>(C->dlist + cl.shot_w), inv_s2, C->dpred, C->part, C->nblk,
                       st));
    CK(launch_misfit(nsamp, nsg, C->part, C->nblk, scale * 0.5 * inv_s2, misfit, C->status, st));
    C->launches[1] += 2;
  }
  prof_mark(C, 2, st);

  nv.phase("reverse sweep");
  // reverse sweep: recompute each earlier segment, then the adjoint steps
  const int sh_f = shape_fwd(C);
  StepParams F = base_params(C, B, nsg, sh_f);  // recompute: sources only, no sampling
  F.inj_off = reinterpret_cast<const int*>(C->dlist + cl.inj_off[sh_f]);
  F.inj_bstride = C->ntiles_s[sh_f] + 1;
  F.inj = reinterpret_cast<const int4*>(C->dlist + cl.inj[sh_f]);
  F.series = C->wav;
  F.series_ld = 1;
  StepParams A = base_params(C, B, nsg, sh_a);  // adjoint: residual at receivers, sample sources
  A.inj_off = C->rec_off[sh_a];
  A.inj_bstride = 0;
  A.inj = C->rec_inj[sh_a];
  A.series = C->dpred;
  A.series_bstride = (long long)nt * nr;
  A.series_ld = nr;
  A.smp_off = reinterpret_cast<const int*>(C->dlist + cl.smp_off[sh_a]);
  A.smp_bstride = C->ntiles_s[sh_a] + 1;
  if (C->L.ndim == 3)
    A.smp4 = reinterpret_cast<const int4*>(C->dlist + cl.smp[sh_a]);
  else
    A.smp = reinterpret_cast<const int2*>(C->dlist + cl.smp[sh_a]);
  A.smp_out = C->qsrc;
  A.smp_bstride_out = (long long)nt * C->Emax;
  A.smp_ld = C->Emax;
  long long adj_launch = 0;
  for (int j = plan.jL; j >= 0; j--) {
    if ((rc = run_steps(C, false, F, rc_off[j], rc_n[j], nsamp, B, M, st, &adj_launch)) != FWI_OK) return rc;
    if ((rc = run_steps(C, true, A, ad_off[j], ad_n[j], nsamp, B, M, st, &adj_launch)) != FWI_OK) return rc;
  }
  C->launches[2] += adj_launch;
  prof_mark(C, 3, st);
  nv.phase("source imaging and fold");
  CK(launch_source_imaging(B, nsg, nt, C->Emax, C->qsrc, C->wav,
                           reinterpret_cast<const int*>(C->dlist + cl.src_cnt),
                           reinterpret_cast<const long long*>(C->dlist + cl.src_pos),
                           reinterpret_cast<const float*>(C->dlist + cl.src_amp), C->stmp, C->G, C->L.field,
                           wf_per_acc, st));
  CK(launch_finalize(C->L, vel, C->G, nsamp, nsg / wf_per_acc, scale, grad, st));
  C->launches[3] += 3;
  prof_mark(C, 4, st);
  if (C->prof) {  // accumulate this chunk's phase times
    CK(cudaEventSynchronize(C->ev[4]));
    for (int i = 0; i < 4; i++) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, C->ev[i], C->ev[i + 1]));
      C->prof_ms[i] += ms;
    }
  }
  return FWI_OK;
}

// Shared driver of fwi_gradient (d_obs set) and fwi_adjoint (cot set):
// chunking of the samples, then one gradient_chunk per chunk.
static int gradient_calls(fwi_ctx* C, const float* vel, int nsamp, const int32_t* perm, const int8_t* w,
                          const int32_t* sg, int nsg, const float* d_obs, const float* cot, double sigma_y,
                          double scale, float* grad, double* misfit, cudaStream_t st) {
  Ranges nv(cot ? "fwi_adjoint" : "fwi_gradient");
  const int nt = C->g.nt;
  // Samples per chunk: the whole batch when its checkpoint plan fits the pool,
  // otherwise the chunk size that minimises (chunks) x (2 nt + recomputed
  // steps) x (time of one step).  In 2D all steps of a phase share one launch
  // and a step costs the work of the busiest CTA, ceil(items / SMs) tiles x
  // nsg supergathers (~1.7 us per tile), but at least ~15 us: with about one
  // item per CTA each step waits for its neighbours' previous one (flag,
  // fence, poll, TMA latency); plus ~20 us per launch (three per checkpoint
  // segment).  In 3D a step (a launch of at least ~8 us, or one step of a
  // multi-step launch) runs ceil(CTAs / SMs) waves of equal CTAs (one CTA
  // per SM), each CTA a column of TX3 x TY3 x nzp points at ~16 B per point
  // from a ~6 TB/s share.
  int nsm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 1;
  int best_c = -1;
  double best_cost = 0.0;
  for (int c = nsamp; c >= 1; c--) {
    const size_t slot_bytes = (size_t)C->L.field * c * nsg * 4;
    Plan p;
    if (!make_plan(nt, (long long)(C->pool_bytes / slot_bytes), &p)) continue;
    const int nchunks = (nsamp + c - 1) / c;
    double cost;
    if (C->L.ndim == 2) {
      const double per_cta = std::ceil((double)c * C->ntiles / nsm) * nsg;
      cost = nchunks * ((2.0 * nt + (double)p.recompute) * std::max(per_cta * 1.7e-6, 15e-6) +
                        (1.0 + 2.0 * (p.jL + 1)) * 20e-6);
    } else {
      // CTAs of a step launch: tiles x wavefields (x pairs with pair tiles)
      const int sh = shape_adj(C, nsg);
      const double waves = std::ceil((double)c * nsg / (sh ? 2 : 1) * C->ntiles_s[sh] / nsm);
      const double t_wave = (double)TX3 * TY3 * C->L.nzp * 16.0 / (6e12 / nsm);
      const double t_launch = std::max(8e-6, waves * t_wave);
      cost = nchunks * (2.0 * nt + (double)p.recompute) * t_launch;
    }
    if (best_c < 0 || cost < best_cost * 0.999) {
      best_c = c;
      best_cost = cost;
    }
  }
  if (best_c < 0) return FWI_ERR_OOM;
  for (int i = 0; i < 4; i++) {
    C->launches[i] = 0;
    C->prof_ms[i] = 0.f;
  }
  C->chunk_samples = best_c;
  C->last_was_gradient = true;
  const long long phys = C->L.phys;
  for (int s0 = 0; s0 < nsamp; s0 += best_c) {
    const int n = std::min(best_c, nsamp - s0);
    const size_t rec0 = (size_t)s0 * nsg * nt * C->nr;
    const int rc = gradient_chunk(C, vel + (size_t)s0 * phys, n, perm + (size_t)s0 * C->ns, w + (size_t)s0 * C->ns,
                                  sg, nsg, d_obs, cot ? cot + rec0 : nullptr, sigma_y, scale,
                                  grad + (size_t)s0 * phys, misfit ? misfit + s0 : nullptr, st, best_c * nsg);
    if (rc != FWI_OK) return rc;
  }
  return FWI_OK;
}

int fwi_gradient(fwi_ctx* C, const float* vel, int nsamp, const int32_t* perm, const int8_t* w, const int32_t* sg,
                 int nsg, const float* d_obs, double sigma_y, double scale, float* grad, double* misfit,
                 void* stream) {
  const int rc = validate_call(C, vel, nsamp, perm, w, sg, nsg);
  if (rc != FWI_OK) return rc;
  if (!d_obs || !grad || !misfit || !(sigma_y > 0)) return FWI_ERR_ARG;
  if (!(scale > 0)) {
    long long tot = 0;
    for (int j = 0; j < nsg; j++) tot += sg[j];
    scale = (double)C->ns / (double)tot;
  }
  return gradient_calls(C, vel, nsamp, perm, w, sg, nsg, d_obs, nullptr, sigma_y, scale, grad, misfit,
                        (cudaStream_t)stream);
}

int fwi_adjoint(fwi_ctx* C, const float* vel, int nsamp, const int32_t* perm, const int8_t* w, const int32_t* sg,
                int nsg, const float* d_cot, float* grad, void* stream) {
  const int rc = validate_call(C, vel, nsamp, perm, w, sg, nsg);
  if (rc != FWI_OK) return rc;
  if (!d_cot || !grad) return FWI_ERR_ARG;
  return gradient_calls(C, vel, nsamp, perm, w, sg, nsg, nullptr, d_cot, 1.0, 1.0, grad, nullptr,
                        (cudaStream_t)stream);
}

int langevin_step(float* z, const float* grad, int64_t n, double eta, double nu, double vmin, double vmax,
                  uint64_t seed, uint64_t counter, void* stream) {
  if (!z || !grad || n < 0 || !(vmin <= vmax) || !(eta >= 0) || !(nu >= 0)) return FWI_ERR_ARG;
  if (n == 0) return FWI_OK;
  CK(launch_langevin(z, grad, n, eta, nu, vmin, vmax, seed, counter, (cudaStream_t)stream));
  return FWI_OK;
}

int langevin_step_precond(fwi_ctx* C, float* z, const float* grad, float* v, float* m, int nsamp, double alpha,
                          double beta1, double eps, int64_t k, double eta, double nu, double vmin, double vmax,
                          uint64_t seed, uint64_t counter, void* stream) {
  if (!C || !z || !grad || !v || nsamp < 1 || nsamp > C->max_B || k < 0) return FWI_ERR_ARG;
  if (!(alpha >= 0 && alpha <= 1) || !(eps >= 0) || !(eta >= 0) || !(nu >= 0) || !(vmin <= vmax))
    return FWI_ERR_ARG;
  if (m && !(beta1 >= 0 && beta1 < 1)) return FWI_ERR_ARG;
  if (k > 0 && !(1.0 - pow(alpha, (double)k) > 0)) return FWI_ERR_ARG;  // alpha = 1 needs k = 0
  CK(launch_langevin_precond(z, grad, v, m, nsamp, C->L.phys, alpha, beta1, eps, k, eta, nu, vmin, vmax, seed,
                             counter, C->part, C->nblk, (cudaStream_t)stream));
  return FWI_OK;
}

int renoise(float* x_prev, const float* x_t, const float* x0, int64_t n, double abar_t, double abar_prev,
            double beta_t, uint64_t seed, uint64_t counter, void* stream) {
  if (!x_prev || !x_t || !x0 || n < 0) return FWI_ERR_ARG;
  if (!(abar_t >= 0 && abar_t < 1) || !(abar_prev > 0 && abar_prev <= 1) || !(beta_t > 0 && beta_t < 1))
    return FWI_ERR_ARG;
  if (fabs(abar_t - abar_prev * (1.0 - beta_t)) > 1e-9) return FWI_ERR_ARG;
  if (n == 0) return FWI_OK;
  const double c0 = sqrt(abar_prev) * beta_t / (1.0 - abar_t);
  const double ct = sqrt(1.0 - beta_t) * (1.0 - abar_prev) / (1.0 - abar_t);
  const double sd = sqrt((1.0 - abar_prev) / (1.0 - abar_t) * beta_t);
  CK(launch_renoise(x_prev, x_t, x0, n, c0, ct, sd, seed, counter, (cudaStream_t)stream));
  return FWI_OK;
}

int smooth_prior_grad(fwi_ctx* C, const float* z, const float* zref, int nsamp, double lam, double mu, float* grad,
                      void* stream) {
  if (!C || !z || !zref || !grad || nsamp < 1 || !(lam >= 0) || !(mu >= 0)) return FWI_ERR_ARG;
  CK(launch_prior(C->L, z, zref, nsamp, lam, mu, C->g.hz, C->g.ndim == 3 ? C->g.hy : 1.0, C->g.hx, grad,
                  (cudaStream_t)stream));
  return FWI_OK;
}

int fwi_last_device_status(fwi_ctx* C, void* stream) {
  if (!C) return FWI_ERR_ARG;
  int v = 0;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(&v, C->status, 4, cudaMemcpyDeviceToHost));
  CK(cudaMemset(C->status, 0, 4));
  return v;
}

int fwi_checkpoint_schedule(int nt, int64_t slots, int32_t* desc_out, int cap, int* nsteps, int* segment_len,
                            int* nsegments, int64_t* recomputed, int* slots_used) {
  if (nt <= 0 || !nsteps) return FWI_ERR_ARG;
  Plan plan;
  if (!make_plan(nt, (long long)slots, &plan)) return FWI_ERR_OOM;
  std::vector<StepDesc> d;
  std::vector<int> rc_off, rc_n, ad_off, ad_n;
  gradient_descs(plan, nt, d, rc_off, rc_n, ad_off, ad_n);
  *nsteps = (int)d.size();
  if (segment_len) *segment_len = plan.K;
  if (nsegments) *nsegments = plan.jL + 1;
  if (recomputed) *recomputed = plan.recompute;
  if (slots_used) *slots_used = plan.slots;
  if (!desc_out) return FWI_OK;
  if (cap < (int)d.size()) return FWI_ERR_ARG;
  // launch of each descriptor, as gradient_chunk issues them
  std::vector<int> launch(d.size(), 0), kind(d.size(), 0);
  int l = 1;
  for (int j = plan.jL; j >= 0; j--) {
    if (rc_n[j] > 0) {
      for (int i = rc_off[j]; i < rc_off[j] + rc_n[j]; i++) launch[i] = l;
      l++;
    }
    for (int i = ad_off[j]; i < ad_off[j] + ad_n[j]; i++) {
      launch[i] = l;
      kind[i] = 1;
    }
    l++;
  }
  for (size_t i = 0; i < d.size(); i++) {
    int32_t* r = desc_out + 7 * i;
    r[0] = launch[i];
    r[1] = kind[i];
    r[2] = d[i].cur;
    r[3] = d[i].prev;
    r[4] = d[i].out;
    r[5] = d[i].snap;
    r[6] = d[i].t;
  }
  return FWI_OK;
}

int fwi_plan_info(fwi_ctx* C, int* K, int* nseg, int64_t* rec, int* used, int* avail) {
  if (!C) return FWI_ERR_ARG;
  if (K) *K = C->plan.K;
  if (nseg) *nseg = C->plan.jL + 1;
  if (rec) *rec = C->plan.recompute;
  if (used) *used = C->plan.slots;
  if (avail) *avail = (int)std::min<long long>(C->slots_avail, 1 << 30);
  return FWI_OK;
}

int fwi_set_kernel_variants(fwi_ctx* C, int fwd, int adj) {
  if (!C) return FWI_ERR_ARG;
  if (fwd >= num_variants(C, false) || adj >= num_variants(C, true)) return FWI_ERR_ARG;
  if (C->L.ndim == 3 && ((fwd >= 0 && (fwd & 16) && !(fwd & 8)) || (adj >= 0 && (adj & 16) && !(adj & 8))))
    return FWI_ERR_ARG;  // multi-step (bit 4) needs the persistent grid (bit 3)
  C->forced[0] = fwd < 0 ? -1 : fwd;
  C->forced[1] = adj < 0 ? -1 : adj;
  C->tuned_B = -1;
  return FWI_OK;
}

int fwi_kernel_variants(fwi_ctx* C, int* fwd, int* adj, const char** fwd_name, const char** adj_name,
                        float* fwd_ms, float* adj_ms, int* nvariants) {
  if (!C) return FWI_ERR_ARG;
  if (fwd) *fwd = C->var[0];
  if (adj) *adj = C->var[1];
  if (fwd_name) *fwd_name = variant_name(C, false, C->var[0]);
  if (adj_name) *adj_name = variant_name(C, true, C->var[1]);
  const int n = std::max(num_variants(C, false), num_variants(C, true));
  if (nvariants) *nvariants = n;
  for (int v = 0; v < n && v < kMaxVariants; v++) {
    if (fwd_ms) fwd_ms[v] = C->tune_ms[0][v];
    if (adj_ms) adj_ms[v] = C->tune_ms[1][v];
  }
  return FWI_OK;
}

int fwi_chunking(fwi_ctx* C, int* samples_per_chunk) {
  if (!C || !samples_per_chunk) return FWI_ERR_ARG;
  *samples_per_chunk = C->chunk_samples;
  return FWI_OK;
}

int fwi_set_profiling(fwi_ctx* C, int on) {
  if (!C) return FWI_ERR_ARG;
  C->prof = on != 0;
  return FWI_OK;
}

int fwi_phase_times(fwi_ctx* C, float* ms, int64_t* launches) {
  if (!C || !C->prof) return FWI_ERR_ARG;
  CK(cudaEventSynchronize(C->ev[4]));
  for (int i = 0; i < 4; i++) {
    if (ms) {
      if (C->last_was_gradient) {
        ms[i] = C->prof_ms[i];
      } else {
        CK(cudaEventElapsedTime(&ms[i], C->ev[i], C->ev[i + 1]));
      }
    }
    if (launches) launches[i] = C->launches[i];
  }
  return FWI_OK;
}

}  // extern "C"
