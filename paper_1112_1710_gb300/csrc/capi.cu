// capi.cu -- the C ABI of include/mhd_gpu.h: argument checks, the context
// (scratch arena, status word, device copies of descriptor tables), and the
// dispatch to the kernel translation units.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <memory>
#include <vector>

#include "amr.h"
#include "common.cuh"
#include "launch.h"
#include "regrid.h"
#include "mhd_gpu.h"

using namespace mhd;

namespace {

// A device copy of a small host table, keyed by its bytes.  Entries are
// immutable once uploaded, so a launch may still be reading one while the
// host prepares the next call; repeated calls with the same descriptors
// (every step of a static hierarchy) upload nothing.
struct TableEntry {
  std::vector<char> bytes;
  void* dev = nullptr;
};

uint64_t fnv1a(const void* p, size_t n) {
  const unsigned char* c = (const unsigned char*)p;
  uint64_t h = 1469598103934665603ULL;
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ULL;
  }
  return h;
}

}  // namespace

struct mhd_ctx {
  mhd_params prm;
  int device = 0;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  double* partials = nullptr;
  size_t partials_n = 0;
  int* d_status = nullptr;
  unsigned long long* d_counter = nullptr;  // fallback counter of mhd_prolong_new
  unsigned long long* d_floors = nullptr;   // cells raised by the pressure floor
  void* rflags = nullptr;                   // refluxing's element flags, zero between calls
  size_t rflags_bytes = 0;
  std::string err;
  std::unordered_multimap<uint64_t, TableEntry> tables;
  size_t table_bytes = 0;
  int64_t launches = 0;
  // advance path per element type (index MHD_F64 / MHD_F32) as picked by the
  // autotuner: staged or fused, the fused variant and its z-chunk length (0:
  // chosen per call); staged until the autotuner measured otherwise
  bool use_fused[2] = {false, false};
  bool pred_tiled[2] = {false, false};  // staged path: the shared-memory-tiled predictor
  bool use_pf[2] = {false, false};      // the fused primitive / predictor / Riemann pass
  int pf_variant[2] = {0, 0};           // its shape
  int fused_variant[2] = {0, 0};
  int fused_chunk[2] = {0, 0};
  // per-kernel event timer
  bool timing = false;
  struct Mark {
    int kernel;
    cudaEvent_t start, stop;
  };
  std::vector<Mark> marks;
  double kernel_ms[K_COUNT] = {};
  int64_t kernel_n[K_COUNT] = {};
  KernelTimer timer{};
};

namespace {

constexpr size_t kTableCacheLimit = size_t(256) << 20;

mhd_status fail(mhd_ctx* c, mhd_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

mhd_status cuda_fail(mhd_ctx* c, cudaError_t e, const char* what) {
  return fail(c, MHD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Returns a device pointer holding `n` bytes equal to `host`.
mhd_status table(mhd_ctx* c, const void* host, size_t n, void** out) {
  if (n == 0) {
    *out = nullptr;
    return MHD_OK;
  }
  const uint64_t h = fnv1a(host, n);
  auto range = c->tables.equal_range(h);
  for (auto it = range.first; it != range.second; ++it) {
    if (it->second.bytes.size() == n && std::memcmp(it->second.bytes.data(), host, n) == 0) {
      *out = it->second.dev;
      return MHD_OK;
    }
  }
  if (c->table_bytes + n > kTableCacheLimit) {
    // drop every cached table; launches in flight may still read them
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "table cache flush");
    for (auto& kv : c->tables) cudaFree(kv.second.dev);
    c->tables.clear();
    c->table_bytes = 0;
  }
  TableEntry t;
  t.bytes.assign((const char*)host, (const char*)host + n);
  cudaError_t e = cudaMalloc(&t.dev, n);
  if (e != cudaSuccess) return fail(c, MHD_ENOMEM, "table alloc of %zu bytes: %s", n, cudaGetErrorString(e));
  // synchronous copy: the entry is immutable from here on
  e = cudaMemcpy(t.dev, host, n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(t.dev);
    return cuda_fail(c, e, "table upload");
  }
  *out = t.dev;
  c->table_bytes += n;
  c->tables.emplace(h, std::move(t));
  return MHD_OK;
}

mhd_status ensure_scratch(mhd_ctx* c, size_t bytes) {
  if (bytes <= c->scratch_bytes) return MHD_OK;
  if (c->scratch) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "scratch resize");
    cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  cudaError_t e = cudaMalloc(&c->scratch, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, MHD_ENOMEM, "scratch alloc of %zu bytes: %s", want, cudaGetErrorString(e));
  }
  c->scratch_bytes = want;
  return MHD_OK;
}

mhd_status ensure_partials(mhd_ctx* c, size_t n) {
  if (n <= c->partials_n) return MHD_OK;
  if (c->partials) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "partials resize");
    cudaFree(c->partials);
    c->partials = nullptr;
  }
  cudaError_t e = cudaMalloc(&c->partials, n * 8 * sizeof(double));
  if (e != cudaSuccess) return fail(c, MHD_ENOMEM, "partials alloc: %s", cudaGetErrorString(e));
  c->partials_n = n;
  return MHD_OK;
}

size_t elem_size(int dtype) { return dtype == MHD_F64 ? 8 : 4; }

// Host checks of one descriptor and its conversion to the device form.
mhd_status convert(mhd_ctx* c, const mhd_patch_desc& d, int idx, DPatch& o) {
  if (d.dtype != MHD_F64 && d.dtype != MHD_F32)
    return fail(c, MHD_EINVAL, "patch %d (id %d): dtype %d", idx, d.patch_id, d.dtype);
  if (d.nghost < 0 || d.nghost > 64)
    return fail(c, MHD_EINVAL, "patch %d (id %d): nghost %d", idx, d.patch_id, d.nghost);
  if (d.stride[0] != 1)
    return fail(c, MHD_EINVAL, "patch %d (id %d): stride[0] must be 1", idx, d.patch_id);
  std::memset(&o, 0, sizeof o);
  int64_t N[3];
  for (int a = 0; a < 3; ++a) {
    int64_t n = (int64_t)d.interior.hi[a] - d.interior.lo[a] + 1;
    if (n < 1 || n > (1 << 20))
      return fail(c, MHD_EINVAL, "patch %d (id %d): empty or huge interior along axis %d", idx, d.patch_id, a);
    N[a] = n + 2 * d.nghost;
    o.n[a] = (int32_t)n;
    o.N[a] = (int32_t)N[a];
    o.glo[a] = d.interior.lo[a] - d.nghost;
    if (!(d.dx[a] > 0.0))
      return fail(c, MHD_EINVAL, "patch %d (id %d): dx[%d] must be > 0", idx, d.patch_id, a);
    o.dx[a] = d.dx[a];
    o.dxf[a] = (float)d.dx[a];
    o.rdx[a] = 1.0 / d.dx[a];
  }
  if (d.stride[1] < N[0] + 1 || d.stride[2] < d.stride[1] * (N[1] + 1))
    return fail(c, MHD_EINVAL, "patch %d (id %d): strides too small for the face arrays", idx, d.patch_id);
  if (N[0] * N[1] * N[2] > (int64_t)1 << 31)
    return fail(c, MHD_EINVAL, "patch %d (id %d): more than 2^31 cells", idx, d.patch_id);
  for (int q = 0; q < 5; ++q) {
    if (!d.U[q]) return fail(c, MHD_EINVAL, "patch %d (id %d): U[%d] is NULL", idx, d.patch_id, q);
    o.U[q] = d.U[q];
  }
  for (int a = 0; a < 3; ++a) {
    if (!d.B[a]) return fail(c, MHD_EINVAL, "patch %d (id %d): B[%d] is NULL", idx, d.patch_id, a);
    o.B[a] = d.B[a];
  }
  o.s1 = d.stride[1];
  o.s2 = d.stride[2];
  o.nelem = d.stride[2] * (N[2] + 1);
  o.snelem = (o.nelem + 7) / 8 * 8;
  o.g = d.nghost;
  o.dt_scale = 1.0;
  o.cfl_scale = 1.0;
  return MHD_OK;
}

mhd_status begin(mhd_ctx* c) {
  if (!c) return MHD_EINVAL;
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
  return MHD_OK;
}

// block table over a per-patch element count
void tasks_for(const std::vector<int64_t>& counts, std::vector<BlockTask>& out) {
  out.clear();
  for (size_t p = 0; p < counts.size(); ++p)
    for (int64_t s = 0; s < counts[p]; s += kThreads) out.push_back(BlockTask{(int32_t)p, (int32_t)s});
}

// Block table (list_elem) of items with counts[i] >= 1 elements each, packed
// (small items share blocks) or aligned to the items, uploaded to the
// context's table cache.  Measured on the AMR hierarchies: packing pays for
// lists of many small boxes (prolongation, restriction, the top layers of
// ghost copies) and costs for lists whose boxes fill their blocks (copies,
// flux-register captures), where threads of one block then read different
// items.
mhd_status packed_table(mhd_ctx* c, const std::vector<int64_t>& counts, bool packed, PackedTasks& out) {
  std::vector<int64_t> starts(counts.size() + 1, 0);
  for (size_t i = 0; i < counts.size(); ++i) starts[i + 1] = starts[i] + counts[i];
  std::vector<BlockTask> tasks;
  if (packed) {
    size_t item = 0;
    for (int64_t b = 0; b < starts.back(); b += kThreads) {
      while (starts[item + 1] <= b) ++item;
      tasks.push_back(BlockTask{(int32_t)item, (int32_t)(b - starts[item])});
    }
  } else {
    tasks_for(counts, tasks);
  }
  if (tasks.size() > 0x7fffffff || counts.size() > 0x7fffffff) return fail(c, MHD_EINVAL, "launch too large");
  void *d_t = nullptr, *d_s = nullptr;
  mhd_status r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t);
  if (!r) r = table(c, starts.data(), starts.size() * sizeof(int64_t), &d_s);
  if (r) return r;
  out.tasks = (const BlockTask*)d_t;
  out.starts = (const int64_t*)d_s;
  out.nblocks = (int)tasks.size();
  out.nitems = (int)counts.size();
  out.packed = packed ? 1 : 0;
  return MHD_OK;
}

// Counts of the top-layer items (box i, axis a) -> item 3 i + a: the box's
// extent over the two transverse axes.
std::vector<int64_t> top_counts(const std::vector<std::array<int32_t, 3>>& ext) {
  const size_t n = ext.size();
  std::vector<int64_t> out(3 * n);
  for (size_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) out[3 * i + a] = (int64_t)ext[i][(a + 1) % 3] * ext[i][(a + 2) % 3];
  return out;
}

// Block tables of the staged advance: over each patch's UB+2 (t2), the
// predictor / flux region (t1) and the update region (tu) of an element of
// `elem` bytes; UB = interior grown by the patch's k.
void staged_tasks(const std::vector<DPatch>& dp, size_t elem, std::vector<BlockTask>& t2,
                  std::vector<BlockTask>& t1, std::vector<BlockTask>& tu) {
  const size_t n = dp.size();
  const int m1 = region_m1(elem), mu = region_mu(elem) + region_mu_top(elem);
  std::vector<int64_t> c2(n), c1(n), cu(n);
  for (size_t p = 0; p < n; ++p) {
    int64_t v2 = 1, v1 = 1, vu = 1;
    for (int d = 0; d < 3; ++d) {
      const int64_t e = dp[p].n[d] + 2 * dp[p].k;
      v2 *= e + 4;
      v1 *= e + 2 * m1;
      vu *= e + mu;
    }
    c2[p] = v2;
    c1[p] = v1;
    cu[p] = vu;
  }
  tasks_for(c2, t2);
  tasks_for(c1, t1);
  tasks_for(cu, tu);
}

double eps_for(const mhd_params& prm, int dtype) {
  if (prm.upwind_eps > 0.0) return prm.upwind_eps;
  return dtype == MHD_F64 ? 1e-10 : 1e-5;
}

void timer_mark(void* self, int kernel, int phase, cudaStream_t s) {
  mhd_ctx* c = (mhd_ctx*)self;
  if (phase == 0) {
    mhd_ctx::Mark m{kernel, nullptr, nullptr};
    cudaEventCreate(&m.start);
    cudaEventCreate(&m.stop);
    cudaEventRecord(m.start, s);
    c->marks.push_back(m);
  } else {
    cudaEventRecord(c->marks.back().stop, s);
  }
}

const KernelTimer* timer_of(mhd_ctx* c) { return c->timing ? &c->timer : nullptr; }

const char* const kKernelNames[K_COUNT] = {"k_prim",  "k_pred",    "k_edge",     "k_flux",   "k_emf",
                                            "k_update", "k_cfl",     "k_ghost",    "k_sums",   "k_reflux",
                                            "k_fused",  "k_commit",  "k_prolong",  "k_restrict", "k_capture",
                                            "k_pf"};

// converts a descriptor array (all of one dtype) to device form
mhd_status convert_all(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, std::vector<DPatch>& dp,
                       int* dtype) {
  if (n < 0 || (n > 0 && !patches)) return fail(c, MHD_EINVAL, "bad patch array");
  dp.resize(n);
  for (int p = 0; p < n; ++p) {
    mhd_status r = convert(c, patches[p], p, dp[p]);
    if (r) return r;
    if (p == 0 && *dtype < 0) *dtype = patches[0].dtype;
    if (patches[p].dtype != *dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
  }
  return MHD_OK;
}

}  // namespace

extern "C" {

const char* mhd_version(void) {
  return "mhdgpu 0.1 sm_103a (fp64 --fmad=false, fp32 --fmad=true)";
}

mhd_status mhd_ctx_create(const mhd_params* params, int32_t device, mhd_ctx** out) {
  if (!out) return MHD_EINVAL;
  *out = nullptr;
  if (!params || !(params->gamma > 1.0) || !(params->cfl > 0.0) || params->cfl > 1.0 ||
      params->limiter < 0 || params->limiter > 2 || params->emf < 0 || params->emf > 1 ||
      params->fp64_contract < 0 || params->fp64_contract > 1 || params->advance_kernel < 0 ||
      params->advance_kernel > 4 || params->fused_chunk < 0 || params->kernel_shape < 0 ||
      params->kernel_shape > 16 || !(params->p_floor >= 0.0) ||
      !(params->rho_floor >= 0.0))
    return MHD_EINVAL;
  mhd_ctx* c = new mhd_ctx();
  c->prm = *params;
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_floors, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_floors, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_floors) cudaFree(c->d_floors);
    delete c;
    return MHD_ECUDA;
  }
  *out = c;
  return MHD_OK;
}

mhd_status mhd_ctx_clone(const mhd_ctx* src, mhd_ctx** out) {
  if (!out) return MHD_EINVAL;
  *out = nullptr;
  if (!src) return MHD_EINVAL;
  mhd_ctx* c = nullptr;
  mhd_status r = mhd_ctx_create(&src->prm, src->device, &c);
  if (r) return r;
  for (int i = 0; i < 2; ++i) {
    c->use_fused[i] = src->use_fused[i];
    c->pred_tiled[i] = src->pred_tiled[i];
    c->use_pf[i] = src->use_pf[i];
    c->pf_variant[i] = src->pf_variant[i];
    c->fused_variant[i] = src->fused_variant[i];
    c->fused_chunk[i] = src->fused_chunk[i];
  }
  *out = c;
  return MHD_OK;
}

void mhd_ctx_destroy(mhd_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (auto& kv : c->tables) cudaFree(kv.second.dev);
  if (c->scratch) cudaFree(c->scratch);
  if (c->partials) cudaFree(c->partials);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_counter) cudaFree(c->d_counter);
  if (c->d_floors) cudaFree(c->d_floors);
  if (c->rflags) cudaFree(c->rflags);
  delete c;
}

const char* mhd_last_error(const mhd_ctx* c) {
  return c ? c->err.c_str() : "no context";
}

int64_t mhd_launch_count(const mhd_ctx* c) { return c ? c->launches : 0; }

mhd_status mhd_timing_enable(mhd_ctx* c, int32_t on) {
  mhd_status r = begin(c);
  if (r) return r;
  c->timing = on != 0;
  c->timer.self = c;
  c->timer.mark = timer_mark;
  return MHD_OK;
}

mhd_status mhd_timing_read(mhd_ctx* c, int32_t kernel, double* total_ms, int64_t* launches) {
  mhd_status r = begin(c);
  if (r) return r;
  if (kernel < 0 || kernel >= K_COUNT || !total_ms || !launches) return fail(c, MHD_EINVAL, "bad kernel id");
  for (auto& m : c->marks) {
    cudaError_t e = cudaEventSynchronize(m.stop);
    if (e != cudaSuccess) return cuda_fail(c, e, "timing event");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m.start, m.stop);
    c->kernel_ms[m.kernel] += ms;
    c->kernel_n[m.kernel] += 1;
    cudaEventDestroy(m.start);
    cudaEventDestroy(m.stop);
  }
  c->marks.clear();
  *total_ms = c->kernel_ms[kernel];
  *launches = c->kernel_n[kernel];
  return MHD_OK;
}

mhd_status mhd_timing_reset(mhd_ctx* c) {
  mhd_status r = begin(c);
  if (r) return r;
  double ms;
  int64_t n;
  if ((r = mhd_timing_read(c, 0, &ms, &n))) return r;
  for (int k = 0; k < K_COUNT; ++k) {
    c->kernel_ms[k] = 0.0;
    c->kernel_n[k] = 0;
  }
  return MHD_OK;
}

const char* mhd_kernel_name(int32_t kernel) {
  return (kernel >= 0 && kernel < K_COUNT) ? kKernelNames[kernel] : "";
}

mhd_status mhd_get_device_status(mhd_ctx* c, int32_t* out) {
  mhd_status r = begin(c);
  if (r) return r;
  if (!out) return fail(c, MHD_EINVAL, "out is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "device status sync");
  int v = 0;
  e = cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(c, e, "device status read");
  *out = v;
  return MHD_OK;
}

// Planes per z-chunk of the fused advance: the largest length whose work
// (including the two-plane pipeline start of every chunk) spreads over the
// device's resident CTAs with the smallest estimated makespan, i.e. total
// work / CTAs + one item.
int fused_chunk_auto(const std::vector<DPatch>& dp, int bx, int by, int ctas) {
  static const int cand[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256};
  int best = 8;
  double best_t = 1e300;
  for (int cz : cand) {
    double work = 0.0;
    int zmax = 0;
    for (const DPatch& p : dp) {
      const int ux = p.n[0] + 2 * p.k, uy = p.n[1] + 2 * p.k, uz = p.n[2] + 2 * p.k;
      const int tiles = ((ux + bx - 1) / bx) * ((uy + by - 1) / by);
      const int nch = (uz + cz - 1) / cz;
      work += (double)tiles * (uz + 3.0 * nch);
      zmax = uz > zmax ? uz : zmax;
    }
    const double t = work / ctas + (cz < zmax ? cz : zmax) + 3.0;
    if (t < best_t - 1e-9) {
      best_t = t;
      best = cz;
    }
  }
  return best;
}

const FusedVariant& fused_variant_of(int dtype, int v) {
  return dtype == MHD_F32 ? kFusedVariants32[v] : kFusedVariants64[v];
}

// Work items (x-y tiles x z-chunks, largest first) and k_commit blocks of a
// fused call.
void fused_items(const std::vector<DPatch>& dp, int bx, int by, int cz, std::vector<FusedItem>& items,
                 std::vector<BlockTask>& ctasks) {
  items.clear();
  std::vector<int64_t> ccnt(dp.size());
  for (size_t p = 0; p < dp.size(); ++p) {
    const DPatch& q = dp[p];
    const int lo = q.g - q.k;
    const int ux = q.n[0] + 2 * q.k, uy = q.n[1] + 2 * q.k, uz = q.n[2] + 2 * q.k;
    for (int z0 = 0; z0 < uz; z0 += cz)
      for (int y0 = 0; y0 < uy; y0 += by)
        for (int x0 = 0; x0 < ux; x0 += bx) {
          FusedItem it{};
          it.patch = (int32_t)p;
          it.x0 = lo + x0;
          it.y0 = lo + y0;
          it.z0 = lo + z0;
          it.z1 = lo + (z0 + cz < uz ? z0 + cz : uz);
          items.push_back(it);
        }
    ccnt[p] = (int64_t)(ux + 1) * (uy + 1) * (uz + 1);
  }
  // largest items first (longest chunks, widest tiles), so the queue ends on short ones
  const auto work = [&](const FusedItem& w) {
    const DPatch& q = dp[w.patch];
    const int hx = q.g + q.n[0] + q.k, hy = q.g + q.n[1] + q.k;
    const int tx = hx - w.x0 < bx ? hx - w.x0 : bx, ty = hy - w.y0 < by ? hy - w.y0 : by;
    return (int64_t)(tx + 2) * (ty + 2) * (w.z1 - w.z0 + 3);
  };
  std::stable_sort(items.begin(), items.end(),
                   [&](const FusedItem& u, const FusedItem& v) { return work(u) > work(v); });
  tasks_for(ccnt, ctasks);
}

// Work items of the fused primitive / predictor / Riemann pass: x-y tiles of
// at most tx x ty cells over each patch's UB+1 region, the extents along each
// axis as equal as the cell count allows, and chunks of cz of its planes.
void pf_items(const std::vector<DPatch>& dp, int tx, int ty, int cz, std::vector<FusedItem>& items) {
  items.clear();
  for (size_t p = 0; p < dp.size(); ++p) {
    const DPatch& q = dp[p];
    const int lo = q.g - q.k - 1;
    const int ex = q.n[0] + 2 * q.k + 2, ey = q.n[1] + 2 * q.k + 2, ez = q.n[2] + 2 * q.k + 2;
    const int nx = (ex + tx - 1) / tx, ny = (ey + ty - 1) / ty;
    for (int z0 = 0; z0 < ez; z0 += cz)
      for (int j = 0, y0 = 0; j < ny; ++j) {
        const int wy = ey / ny + (j < ey % ny ? 1 : 0);
        for (int i = 0, x0 = 0; i < nx; ++i) {
          const int wx = ex / nx + (i < ex % nx ? 1 : 0);
          FusedItem it{};
          it.patch = (int32_t)p;
          it.x0 = lo + x0;
          it.y0 = lo + y0;
          it.z0 = lo + z0;
          it.z1 = lo + (z0 + cz < ez ? z0 + cz : ez);
          it.tx = wx;
          it.ty = wy;
          items.push_back(it);
          x0 += wx;
        }
        y0 += wy;
      }
  }
}

// One block per tile of each patch's UB+1 for the tiled predictor.
void pred_tiles(const std::vector<DPatch>& dp, int dtype, std::vector<BlockTask>& out) {
  const int* T = dtype == MHD_F32 ? kPredTile32 : kPredTile64;
  out.clear();
  for (size_t p = 0; p < dp.size(); ++p) {
    const DPatch& q = dp[p];
    const int ex = q.n[0] + 2 * q.k + 2, ey = q.n[1] + 2 * q.k + 2, ez = q.n[2] + 2 * q.k + 2;
    const int64_t nt = (int64_t)((ex + T[0] - 1) / T[0]) * ((ey + T[1] - 1) / T[1]) * ((ez + T[2] - 1) / T[2]);
    for (int64_t t = 0; t < nt; ++t) out.push_back(BlockTask{(int32_t)p, (int32_t)t});
  }
}

int sm_count(int dev) {
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
  return nsm;
}

// Host checks of an advance's patch array and their device descriptors.
mhd_status advance_patches(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, const int32_t* grow,
                           const double* dt_scale, std::vector<DPatch>& dp) {
  dp.assign(n, DPatch{});
  const int dtype = patches[0].dtype;
  mhd_status r;
  for (int p = 0; p < n; ++p) {
    if ((r = convert(c, patches[p], p, dp[p]))) return r;
    if (patches[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
    const int k = grow ? grow[p] : 0;
    if (k < 0 || k + 2 > patches[p].nghost)
      return fail(c, MHD_EINVAL, "patch %d (id %d): grow %d needs grow + 2 <= nghost (%d)", p,
                  patches[p].patch_id, k, patches[p].nghost);
    if (dt_scale && !(dt_scale[p] > 0.0)) return fail(c, MHD_EINVAL, "dt_scale[%d] must be > 0", p);
    dp[p].k = k;
    dp[p].dt_scale = dt_scale ? dt_scale[p] : 1.0;
  }
  return MHD_OK;
}

cudaError_t run_advance_args(mhd_ctx* c, int dtype, const AdvanceArgs& a, cudaStream_t s) {
  return dtype == MHD_F32           ? advance_f32(a, s)
         : c->prm.fp64_contract ? advance_f64c(a, s)
                                : advance_f64(a, s);
}

// Checks each flux-register capture of an advance call against the faces /
// edges the call computes, converts it to device form and marks its patch
// (flags bit 0); fused_ok is cleared when a capture needs face fluxes outside
// the update box (the fused kernel stores only those).
static mhd_status scan_captures(mhd_ctx* c, std::vector<DPatch>& dp, const mhd_capture* caps, int32_t ncap,
                                std::vector<DCapture>& dc, std::vector<int64_t>& ccounts, bool& fused_ok) {
  const int n = (int)dp.size();
  dc.resize(ncap);
  ccounts.resize(ncap);
  for (int t = 0; t < ncap; ++t) {
    const mhd_capture& m = caps[t];
    if (m.patch < 0 || m.patch >= n || (m.kind != 0 && m.kind != 1) || m.axis < 0 || m.axis > 2 ||
        (m.mode != 0 && m.mode != 1) || !m.dst)
      return fail(c, MHD_EINVAL, "capture %d: bad patch, kind, axis, mode or dst", t);
    DPatch& p = dp[m.patch];
    DCapture& o = dc[t];
    o.patch = m.patch;
    o.kind = m.kind;
    o.axis = m.axis;
    o.mode = m.mode;
    o.dst = m.dst;
    int64_t cnt = 1;
    for (int d = 0; d < 3; ++d) {
      const int lo = m.box.lo[d] - p.glo[d], hi = m.box.hi[d] - p.glo[d];
      const int ulo = p.g - p.k, uhi = p.g + p.n[d] - 1 + p.k;
      int alo, ahi;  // computed range along d
      if (m.kind == 0) {
        alo = d == m.axis ? ulo : ulo - 1;
        ahi = d == m.axis ? uhi + 1 : uhi + 1;
      } else {
        alo = ulo;
        ahi = d == m.axis ? uhi : uhi + 1;
      }
      if (hi < lo || lo < alo || hi > ahi)
        return fail(c, MHD_EINVAL, "capture %d: box outside the elements the advance computes (axis %d)", t, d);
      // the fused kernel stores the face fluxes of the update box only
      if (m.kind == 0 && d != m.axis && (lo < ulo || hi > uhi)) fused_ok = false;
      o.lo[d] = lo;
      o.ext[d] = hi - lo + 1;
      cnt *= o.ext[d];
    }
    ccounts[t] = cnt;
    p.flags |= 1;
  }
  return MHD_OK;
}

// The advance of mhd_patch_advance; with cfl_dt set (single-level steps, no
// captures), the step first computes its own CFL dt into *d_dt: inside k_prim
// for the staged kernels, by the separate reduction before the fused one.
static mhd_status advance_impl(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, const int32_t* grow,
                        const double* d_dt, const double* dt_scale, const mhd_capture* caps, int32_t ncap,
                        void* stream, bool cfl_dt) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 0 || (n > 0 && !patches)) return fail(c, MHD_EINVAL, "bad patch array");
  if (!d_dt) return fail(c, MHD_EINVAL, "d_dt is NULL");
  if (ncap < 0 || (ncap > 0 && !caps)) return fail(c, MHD_EINVAL, "bad capture list");
  if (n == 0) return MHD_OK;
  std::vector<DPatch> dp;
  const int dtype = patches[0].dtype;
  if ((r = advance_patches(c, patches, n, grow, dt_scale, dp))) return r;
  // which advance: the context's (autotuned) choice, or forced staged / fused
  bool fused = c->prm.advance_kernel == 2 || (c->prm.advance_kernel == 0 && c->use_fused[dtype == MHD_F32 ? 1 : 0]);
  const bool pf = !fused && (c->prm.advance_kernel == 4 ||
                             (c->prm.advance_kernel == 0 && c->use_pf[dtype == MHD_F32 ? 1 : 0]));
  if (cfl_dt && (fused || pf)) {
    // neither the fused kernel nor the fused pass has a primitive pass of its
    // own: the CFL reduction runs first
    if ((r = mhd_cfl_dt(c, patches, n, nullptr, const_cast<double*>(d_dt), stream))) return r;
    cfl_dt = false;
  }
  // flux-register captures: checked against the faces / edges this call computes
  std::vector<DCapture> dc(ncap);
  std::vector<int64_t> ccounts(ncap);
  bool fused_ok = true;
  if ((r = scan_captures(c, dp, caps, ncap, dc, ccounts, fused_ok))) return r;
  if (!fused_ok) fused = false;
  // arena: per patch its stage planes (staged) or its output copy, plus the
  // flux planes when it feeds captures (fused); then the step constants, then
  // the work-queue head
  int64_t off = 0;
  for (int p = 0; p < n; ++p) {
    dp[p].scr = off;
    off += (int64_t)((!fused || (dp[p].flags & 1)) ? SC_COUNT : 8) * dp[p].snelem;
  }
  const int64_t stepc_off = off;
  off += 8 * (int64_t)n;
  const size_t es = elem_size(dtype);
  const size_t counter_byte = ((size_t)off * es + 15) / 16 * 16;
  if ((r = ensure_scratch(c, counter_byte + 16))) return r;
  std::vector<BlockTask> tasks, tasks1, tasksu, ptasks;
  std::vector<FusedItem> items;
  std::vector<BlockTask> ctasks;
  const int di = dtype == MHD_F32 ? 1 : 0;
  const int shape = c->prm.kernel_shape > 0 ? c->prm.kernel_shape - 1 : pf ? c->pf_variant[di] : c->fused_variant[di];
  if (shape >= (pf ? (di ? kNumPf32 : kNumPf64) : (di ? kNumFused32 : kNumFused64)))
    return fail(c, MHD_EINVAL, "kernel_shape %d is not compiled for this element type", c->prm.kernel_shape);
  if (pf) {
    staged_tasks(dp, elem_size(dtype), tasks, tasks1, tasksu);
    const PfVariant& pv = di ? kPfVariants32[shape] : kPfVariants64[shape];
    pf_items(dp, pv.tx, pv.ty,
             c->prm.fused_chunk > 0 ? c->prm.fused_chunk : c->fused_chunk[di] > 0 ? c->fused_chunk[di] : 16, items);
    if (items.size() > 0x7fffffff || tasksu.size() > 0x7fffffff) return fail(c, MHD_EINVAL, "launch too large");
  } else if (!fused) {
    staged_tasks(dp, elem_size(dtype), tasks, tasks1, tasksu);
    if (c->prm.advance_kernel == 3 || c->pred_tiled[dtype == MHD_F32 ? 1 : 0]) pred_tiles(dp, dtype, ptasks);
    if (tasks.size() > 0x7fffffff || ptasks.size() > 0x7fffffff) return fail(c, MHD_EINVAL, "launch too large");
  } else {
    const FusedVariant& v = fused_variant_of(dtype, shape);
    const int cz = c->prm.fused_chunk > 0   ? c->prm.fused_chunk
                   : c->fused_chunk[di] > 0 ? c->fused_chunk[di]
                                            : fused_chunk_auto(dp, v.bx, v.by, sm_count(c->device));
    fused_items(dp, v.bx, v.by, cz, items, ctasks);
    if (items.size() > 0x7fffffff) return fail(c, MHD_EINVAL, "launch too large");
  }
  void *d_p = nullptr, *d_t = nullptr, *d_t1 = nullptr, *d_tu = nullptr, *d_i = nullptr, *d_ct = nullptr,
       *d_pt = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  if ((r = table(c, tasks1.data(), tasks1.size() * sizeof(BlockTask), &d_t1))) return r;
  if ((r = table(c, tasksu.data(), tasksu.size() * sizeof(BlockTask), &d_tu))) return r;
  if ((r = table(c, ptasks.data(), ptasks.size() * sizeof(BlockTask), &d_pt))) return r;
  if ((r = table(c, items.data(), items.size() * sizeof(FusedItem), &d_i))) return r;
  if ((r = table(c, ctasks.data(), ctasks.size() * sizeof(BlockTask), &d_ct))) return r;
  AdvanceArgs a{};
  a.patches = (const DPatch*)d_p;
  a.npatches = n;
  a.tasks = (const BlockTask*)d_t;
  a.nblocks = (int)tasks.size();
  a.tasks1 = (const BlockTask*)d_t1;
  a.nblocks1 = (int)tasks1.size();
  a.tasksu = (const BlockTask*)d_tu;
  a.nblocksu = (int)tasksu.size();
  a.ptasks = (const BlockTask*)d_pt;
  a.npblocks = (int)ptasks.size();
  a.scratch = c->scratch;
  a.stepc = (char*)c->scratch + (size_t)stepc_off * es;
  a.gamma = c->prm.gamma;
  a.eps_up = eps_for(c->prm, dtype);
  a.limiter = c->prm.limiter;
  a.emf = c->prm.emf;
  a.d_dt = d_dt;
  a.d_status = c->d_status;
  a.timer = timer_of(c);
  a.fused = fused;
  a.items = (const FusedItem*)d_i;
  a.nitems = (int)items.size();
  a.counter = (int*)((char*)c->scratch + counter_byte);
  a.ctasks = (const BlockTask*)d_ct;
  a.nctasks = (int)ctasks.size();
  a.variant = shape;
  a.commit = true;
  a.cfl_out = cfl_dt ? (unsigned long long*)const_cast<double*>(d_dt) : nullptr;
  a.cfl = c->prm.cfl;
  a.p_floor = c->prm.p_floor;
  a.rho_floor = c->prm.rho_floor;
  a.d_floors = c->d_floors;
  a.pf = pf;
  if (pf) {
    a.pf_items = (const FusedItem*)d_i;
    a.npf = (int)items.size();
    a.fused = false;
  }
  cudaError_t e = run_advance_args(c, dtype, a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "patch advance launch");
  // fused: step constants, k_fused, k_commit; staged with the CFL dt: + reset
  c->launches += (fused ? 3 : pf ? (elem_size(dtype) == 8 ? 4 : 3) : staged_launches(elem_size(dtype)) + (cfl_dt ? 1 : 0)) +
                 (c->prm.p_floor > 0.0 || c->prm.rho_floor > 0.0 ? 1 : 0);
  if (ncap > 0) {
    PackedTasks pc{};
    if ((r = packed_table(c, ccounts, false, pc))) return r;
    void* d_c = nullptr;
    if ((r = table(c, dc.data(), dc.size() * sizeof(DCapture), &d_c))) return r;
    e = capture_launch(dtype, (const DPatch*)d_p, (const DCapture*)d_c, pc, c->scratch, d_dt, timer_of(c),
                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "capture launch");
    c->launches += 1;
  }
  return MHD_OK;
}

mhd_status mhd_patch_advance(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, const int32_t* grow,
                             const double* d_dt, const double* dt_scale, const mhd_capture* caps, int32_t ncap,
                             void* stream) {
  return advance_impl(c, patches, n, grow, d_dt, dt_scale, caps, ncap, stream, false);
}

mhd_status mhd_patch_step_cfl(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, double* d_dt_out,
                              void* stream) {
  if (!c) return MHD_EINVAL;
  if (n < 1 || !patches) return fail(c, MHD_EINVAL, "patch_step_cfl needs at least one patch");
  if (!d_dt_out) return fail(c, MHD_EINVAL, "d_dt_out is NULL");
  return advance_impl(c, patches, n, nullptr, d_dt_out, nullptr, nullptr, 0, stream, true);
}

mhd_status mhd_autotune_advance(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, const int32_t* grow,
                                const mhd_capture* caps, int32_t ncap, const double* d_dt, int32_t reps,
                                int32_t* variant_out, int32_t* chunk_out, float* ms_out, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 1 || !patches || !d_dt || reps < 1 || reps > 1000) return fail(c, MHD_EINVAL, "autotune: bad arguments");
  if (ncap < 0 || (ncap > 0 && !caps)) return fail(c, MHD_EINVAL, "bad capture list");
  std::vector<DPatch> dp;
  const int dtype = patches[0].dtype;
  if ((r = advance_patches(c, patches, n, grow, nullptr, dp))) return r;
  // the captures a real call would make: their patches' extra stores, and
  // whether the fused kernel may run at all
  std::vector<DCapture> dc;
  std::vector<int64_t> ccounts;
  bool fused_ok = true;
  if ((r = scan_captures(c, dp, caps, ncap, dc, ccounts, fused_ok))) return r;
  // arena as for a staged call (the staged candidate needs its 92 planes; the
  // fused ones use the first 8 of them as output copies)
  int64_t off = 0;
  int zmax = 1;
  for (int p = 0; p < n; ++p) {
    dp[p].scr = off;
    off += (int64_t)SC_COUNT * dp[p].snelem;
    const int uz = dp[p].n[2] + 2 * dp[p].k;
    zmax = uz > zmax ? uz : zmax;
  }
  const int64_t stepc_off = off;
  off += 8 * (int64_t)n;
  const size_t es = elem_size(dtype);
  const size_t counter_byte = ((size_t)off * es + 15) / 16 * 16;
  // after the work-queue head: a status word of the candidates' own, so that
  // their checks (on whatever the ghost zones hold) leave the context's alone
  if ((r = ensure_scratch(c, counter_byte + 32))) return r;
  std::vector<BlockTask> tasks, tasks1, tasksu, ptasks;
  staged_tasks(dp, elem_size(dtype), tasks, tasks1, tasksu);
  pred_tiles(dp, dtype, ptasks);
  if (tasks.size() > 0x7fffffff || ptasks.size() > 0x7fffffff) return fail(c, MHD_EINVAL, "launch too large");
  void *d_p = nullptr, *d_t = nullptr, *d_t1 = nullptr, *d_tu = nullptr, *d_pt = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  if ((r = table(c, tasks1.data(), tasks1.size() * sizeof(BlockTask), &d_t1))) return r;
  if ((r = table(c, tasksu.data(), tasksu.size() * sizeof(BlockTask), &d_tu))) return r;
  if ((r = table(c, ptasks.data(), ptasks.size() * sizeof(BlockTask), &d_pt))) return r;
  // the fused kernel's copy-back goes to planes of the scratch arena the
  // fused kernel does not use (the predicted-state planes), so that it is
  // timed without touching the patch state
  std::vector<DPatch> dpc = dp;
  const size_t es0 = elem_size(dtype);
  for (int p = 0; p < n; ++p) {
    for (int q = 0; q < 5; ++q) dpc[p].U[q] = (char*)c->scratch + (size_t)(dp[p].scr + (SC_WF + q) * dp[p].snelem) * es0;
    for (int a = 0; a < 3; ++a)
      dpc[p].B[a] = (char*)c->scratch + (size_t)(dp[p].scr + (SC_WF + 5 + a) * dp[p].snelem) * es0;
  }
  void* d_pc = nullptr;
  if ((r = table(c, dpc.data(), dpc.size() * sizeof(DPatch), &d_pc))) return r;
  const int di = dtype == MHD_F32 ? 1 : 0;
  const int nv = fused_ok ? (dtype == MHD_F32 ? kNumFused32 : kNumFused64) : 0;
  const int nsm = sm_count(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(c, e, "autotune events");
  }
  // candidates (choice code, chunk): the fused pass in every shape (-3 - s)
  // x chunk length; the staged kernels with the untiled (-2) and the tiled
  // (-1) predictor; the fused kernel in every shape (s) x chunk length
  std::vector<std::pair<int, int>> cand;
  const int npv = dtype == MHD_F32 ? kNumPf32 : kNumPf64;
  for (int sv = 0; sv < npv; ++sv) {
    std::vector<int> chunks;
    for (int cz : {6, 8, 12, 16, 24, 33}) {
      cz = cz > zmax + 2 ? zmax + 2 : cz;
      if (std::find(chunks.begin(), chunks.end(), cz) == chunks.end()) chunks.push_back(cz);
    }
    for (int cz : chunks) cand.push_back({-3 - sv, cz});
  }
  cand.push_back({-2, 0});
  cand.push_back({-1, 0});
  for (int v = 0; v < nv; ++v) {
    const FusedVariant& fv = fused_variant_of(dtype, v);
    std::vector<int> chunks;
    for (int cz : {fused_chunk_auto(dp, fv.bx, fv.by, nsm), 4, 8, 16, 32, 64}) {
      cz = cz > zmax ? zmax : cz;
      if (std::find(chunks.begin(), chunks.end(), cz) == chunks.end()) chunks.push_back(cz);
    }
    for (int cz : chunks) cand.push_back({v, cz});
  }
  float best = 3.4e38f;
  int bv = 0, bcz = 0;
  bool any = false;
  std::vector<FusedItem> items;
  std::vector<BlockTask> ctasks;
  int skip_shape = -1000;  // a shape this device cannot run: its other chunks are skipped
  for (const auto& cv : cand) {
    const int v = cv.first, cz = cv.second;
    if (v == skip_shape) continue;
    AdvanceArgs a{};
    a.patches = (const DPatch*)d_p;
    a.npatches = n;
    a.tasks = (const BlockTask*)d_t;
    a.nblocks = (int)tasks.size();
    a.tasks1 = (const BlockTask*)d_t1;
    a.nblocks1 = (int)tasks1.size();
    a.tasksu = (const BlockTask*)d_tu;
    a.nblocksu = (int)tasksu.size();
    a.scratch = c->scratch;
    a.stepc = (char*)c->scratch + (size_t)stepc_off * es;
    a.gamma = c->prm.gamma;
    a.eps_up = eps_for(c->prm, dtype);
    a.limiter = c->prm.limiter;
    a.emf = c->prm.emf;
    a.d_dt = d_dt;
    a.d_status = (int*)((char*)c->scratch + counter_byte + 16);
    a.timer = nullptr;
    a.p_floor = c->prm.p_floor;  // the primitives' floors, as in a real call
    a.rho_floor = c->prm.rho_floor;
    a.d_floors = c->d_floors;
    a.commit = false;  // every candidate leaves the patch state as it is
    a.fused = v >= 0;
    if (v == -1) {
      a.ptasks = (const BlockTask*)d_pt;
      a.npblocks = (int)ptasks.size();
    }
    if (v <= -3) {
      const PfVariant& pv = dtype == MHD_F32 ? kPfVariants32[-3 - v] : kPfVariants64[-3 - v];
      pf_items(dp, pv.tx, pv.ty, cz, items);
      void* d_i = nullptr;
      if ((r = table(c, items.data(), items.size() * sizeof(FusedItem), &d_i))) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
      }
      a.pf = true;
      a.pf_items = (const FusedItem*)d_i;
      a.npf = (int)items.size();
      a.variant = -3 - v;
    }
    if (a.fused) {
      const FusedVariant& fv = fused_variant_of(dtype, v);
      fused_items(dp, fv.bx, fv.by, cz, items, ctasks);
      void *d_i = nullptr, *d_ct = nullptr;
      if ((r = table(c, items.data(), items.size() * sizeof(FusedItem), &d_i)) ||
          (r = table(c, ctasks.data(), ctasks.size() * sizeof(BlockTask), &d_ct))) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return r;
      }
      a.items = (const FusedItem*)d_i;
      a.nitems = (int)items.size();
      a.counter = (int*)((char*)c->scratch + counter_byte);
      a.ctasks = (const BlockTask*)d_ct;
      a.nctasks = (int)ctasks.size();
      a.variant = v;
      a.commit_patches = (const DPatch*)d_pc;
    }
    e = run_advance_args(c, dtype, a, s);
    if (e != cudaSuccess) {  // a shape this device cannot run: skip it
      cudaGetLastError();
      skip_shape = v;
      continue;
    }
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = run_advance_args(c, dtype, a, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(c, e, "autotune run");
    }
    c->launches += (a.fused ? 3 : a.pf ? (es == 8 ? 4 : 3) : staged_launches(es)) * (reps + 1);
    ms /= reps;
    if (ms < best) {
      best = ms;
      bv = v;
      bcz = cz;
      any = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!any) return fail(c, MHD_ECUDA, "autotune: no advance ran on this device");
  c->use_fused[di] = bv >= 0;
  c->use_pf[di] = bv <= -3;
  if (bv == -2 || bv == -1) c->pred_tiled[di] = bv == -1;
  c->fused_variant[di] = bv >= 0 ? bv : 0;
  c->pf_variant[di] = bv <= -3 ? -3 - bv : 0;
  c->fused_chunk[di] = bv >= 0 || bv <= -3 ? bcz : 0;
  if (variant_out) *variant_out = bv;
  if (chunk_out) *chunk_out = bcz;
  if (ms_out) *ms_out = best;
  return MHD_OK;
}

mhd_status mhd_cfl_dt(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, const double* scale,
                      double* d_dt_out, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 1 || !patches) return fail(c, MHD_EINVAL, "cfl_dt needs at least one patch");
  if (!d_dt_out) return fail(c, MHD_EINVAL, "d_dt_out is NULL");
  std::vector<DPatch> dp(n);
  std::vector<int64_t> counts(n);
  const int dtype = patches[0].dtype;
  for (int p = 0; p < n; ++p) {
    if ((r = convert(c, patches[p], p, dp[p]))) return r;
    if (patches[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
    if (scale && !(scale[p] > 0.0)) return fail(c, MHD_EINVAL, "scale[%d] must be > 0", p);
    dp[p].cfl_scale = scale ? scale[p] : 1.0;
    counts[p] = (int64_t)dp[p].n[0] * dp[p].n[1] * dp[p].n[2];
  }
  std::vector<BlockTask> tasks;
  tasks_for(counts, tasks);
  void *d_p = nullptr, *d_t = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  cudaError_t e = cfl_dt_launch(dtype, (const DPatch*)d_p, (const BlockTask*)d_t, (int)tasks.size(),
                                c->prm.gamma, c->prm.cfl, d_dt_out, c->d_status, timer_of(c),
                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cfl_dt launch");
  c->launches += tasks.empty() ? 1 : 2;
  return MHD_OK;
}

mhd_status mhd_transfer_copy(mhd_ctx* c, const mhd_patch_desc* old, int32_t no, const mhd_patch_desc* fresh,
                             int32_t nn, const mhd_transfer_item* items, int32_t ni, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (no < 1 || nn < 1 || !old || !fresh || ni < 0 || (ni > 0 && !items))
    return fail(c, MHD_EINVAL, "transfer_copy: bad arguments");
  if (ni == 0) return MHD_OK;
  std::vector<DPatch> dold(no), dnew(nn);
  const int dtype = old[0].dtype;
  for (int p = 0; p < no; ++p) {
    if ((r = convert(c, old[p], p, dold[p]))) return r;
    if (old[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
  }
  for (int p = 0; p < nn; ++p) {
    if ((r = convert(c, fresh[p], p, dnew[p]))) return r;
    if (fresh[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
  }
  std::vector<DTransfer> it(ni);
  std::vector<int64_t> counts(ni);
  for (int t = 0; t < ni; ++t) {
    const mhd_transfer_item& m = items[t];
    if (m.src < 0 || m.src >= no || m.dst < 0 || m.dst >= nn || m.kind < -1 || m.kind > 2)
      return fail(c, MHD_EINVAL, "transfer item %d: bad patch index or kind", t);
    DTransfer& o = it[t];
    o.src = m.src;
    o.dst = m.dst;
    o.kind = m.kind;
    o.pad = 0;
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.box.lo[a], hi = m.box.hi[a];
      const int top = (m.kind == a) ? 0 : -1;  // face arrays hold one more entry along their normal
      for (const DPatch* P : {&dold[m.src], &dnew[m.dst]})
        if (hi < lo || lo - P->glo[a] < 0 || hi - P->glo[a] > P->N[a] + top)
          return fail(c, MHD_EINVAL, "transfer item %d: box outside the arrays", t);
      o.lo[a] = lo;
      o.ext[a] = hi - lo + 1;
      cnt *= o.ext[a];
    }
    counts[t] = cnt;
  }
  std::vector<BlockTask> tasks;
  tasks_for(counts, tasks);
  void *d_o = nullptr, *d_n = nullptr, *d_i = nullptr, *d_t = nullptr;
  if ((r = table(c, dold.data(), dold.size() * sizeof(DPatch), &d_o))) return r;
  if ((r = table(c, dnew.data(), dnew.size() * sizeof(DPatch), &d_n))) return r;
  if ((r = table(c, it.data(), it.size() * sizeof(DTransfer), &d_i))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  cudaError_t e = transfer_copy_launch(dtype, (const DPatch*)d_o, (const DPatch*)d_n, (const DTransfer*)d_i,
                                       (const BlockTask*)d_t, (int)tasks.size(), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "transfer_copy launch");
  c->launches += 1;
  return MHD_OK;
}

mhd_status mhd_prolong_new(mhd_ctx* c, const mhd_patch_desc* coarse, int32_t nc, const mhd_patch_desc* fine,
                           int32_t nf, const mhd_prolong_new_item* items, int32_t ni, int32_t energy_mode,
                           unsigned long long* d_fallbacks, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (nc < 1 || nf < 1 || !coarse || !fine || ni < 0 || (ni > 0 && !items) || (energy_mode != 0 && energy_mode != 1))
    return fail(c, MHD_EINVAL, "prolong_new: bad arguments");
  if (ni == 0) return MHD_OK;
  std::vector<DPatch> dc(nc), df(nf);
  const int dtype = coarse[0].dtype;
  for (int p = 0; p < nc; ++p) {
    if ((r = convert(c, coarse[p], p, dc[p]))) return r;
    if (coarse[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
  }
  for (int p = 0; p < nf; ++p) {
    if ((r = convert(c, fine[p], p, df[p]))) return r;
    if (fine[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
  }
  std::vector<DProlongNew> it(ni);
  std::vector<int64_t> counts(ni);
  for (int t = 0; t < ni; ++t) {
    const mhd_prolong_new_item& m = items[t];
    if (m.coarse < 0 || m.coarse >= nc || m.fine < 0 || m.fine >= nf || !m.mask)
      return fail(c, MHD_EINVAL, "prolong_new item %d: bad patch index or mask", t);
    const DPatch& C = dc[m.coarse];
    const DPatch& F = df[m.fine];
    DProlongNew& o = it[t];
    o.coarse = m.coarse;
    o.fine = m.fine;
    o.mask = m.mask;
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.box.lo[a], hi = m.box.hi[a];
      // the coarse cells and their neighbours inside the coarse arrays, their
      // children and the children's upper faces inside the fine arrays, the
      // box inside the mask's box
      if (hi < lo || lo - 1 - C.glo[a] < 0 || hi + 1 - C.glo[a] > C.N[a] - 1 || 2 * lo - F.glo[a] < 0 ||
          2 * hi + 2 - F.glo[a] > F.N[a] || lo < m.mask_box.lo[a] || hi > m.mask_box.hi[a])
        return fail(c, MHD_EINVAL, "prolong_new item %d: box outside the arrays or the mask", t);
      o.lo[a] = lo;
      o.ext[a] = hi - lo + 1;
      o.mlo[a] = m.mask_box.lo[a];
      o.mext[a] = m.mask_box.hi[a] - m.mask_box.lo[a] + 1;
      cnt *= o.ext[a];
    }
    counts[t] = cnt;
  }
  unsigned long long* nfall = d_fallbacks;
  if (!nfall) {
    if (!c->d_counter) {
      cudaError_t e = cudaMalloc(&c->d_counter, sizeof(unsigned long long));
      if (e != cudaSuccess) return fail(c, MHD_ENOMEM, "counter: %s", cudaGetErrorString(e));
    }
    nfall = c->d_counter;
  }
  std::vector<BlockTask> tasks;
  tasks_for(counts, tasks);
  void *d_c = nullptr, *d_f = nullptr, *d_i = nullptr, *d_t = nullptr;
  if ((r = table(c, dc.data(), dc.size() * sizeof(DPatch), &d_c))) return r;
  if ((r = table(c, df.data(), df.size() * sizeof(DPatch), &d_f))) return r;
  if ((r = table(c, it.data(), it.size() * sizeof(DProlongNew), &d_i))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  cudaError_t e = prolong_new_launch(dtype, (const DPatch*)d_c, (const DPatch*)d_f, (const DProlongNew*)d_i,
                                     (const BlockTask*)d_t, (int)tasks.size(), energy_mode, nfall,
                                     (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "prolong_new launch");
  c->launches += 1;
  return MHD_OK;
}

mhd_status mhd_floor(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 1 || !patches) return fail(c, MHD_EINVAL, "floor: bad arguments");
  if (!(c->prm.p_floor > 0.0 || c->prm.rho_floor > 0.0)) return MHD_OK;
  std::vector<DPatch> dp(n);
  std::vector<int64_t> counts(n);
  const int dtype = patches[0].dtype;
  for (int p = 0; p < n; ++p) {
    if ((r = convert(c, patches[p], p, dp[p]))) return r;
    if (patches[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
    dp[p].k = 0;
    counts[p] = (int64_t)(dp[p].n[0] + 1) * (dp[p].n[1] + 1) * (dp[p].n[2] + 1);
  }
  std::vector<BlockTask> tasks;
  tasks_for(counts, tasks);
  void *d_p = nullptr, *d_t = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  AdvanceArgs a{};
  a.patches = (const DPatch*)d_p;
  a.npatches = n;
  a.tasksu = (const BlockTask*)d_t;
  a.nblocksu = (int)tasks.size();
  a.gamma = c->prm.gamma;
  a.p_floor = c->prm.p_floor;
  a.rho_floor = c->prm.rho_floor;
  a.d_floors = c->d_floors;
  cudaError_t e = dtype == MHD_F32 ? floor_f32(a, (cudaStream_t)stream) : floor_f64(a, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "floor launch");
  c->launches += 1;
  return MHD_OK;
}

mhd_status mhd_floor_count(mhd_ctx* c, int64_t* out) {
  mhd_status r = begin(c);
  if (r) return r;
  if (!out) return fail(c, MHD_EINVAL, "floor_count: out is NULL");
  unsigned long long v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, c->d_floors, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(c->d_floors, 0, sizeof v);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "floor_count");
  *out = (int64_t)v;
  return MHD_OK;
}

mhd_status mhd_flag_cells(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, double theta, uint8_t* d_flags,
                          void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 1 || !patches || !d_flags || !(theta >= 0.0)) return fail(c, MHD_EINVAL, "flag_cells: bad arguments");
  std::vector<DPatch> dp(n);
  std::vector<int64_t> counts(n), off(n);
  const int dtype = patches[0].dtype;
  int64_t total = 0;
  for (int p = 0; p < n; ++p) {
    if ((r = convert(c, patches[p], p, dp[p]))) return r;
    if (patches[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
    if (patches[p].nghost < 1) return fail(c, MHD_EINVAL, "flag_cells: patch %d needs a ghost layer", p);
    counts[p] = (int64_t)dp[p].n[0] * dp[p].n[1] * dp[p].n[2];
    off[p] = total;
    total += counts[p];
  }
  std::vector<BlockTask> tasks;
  tasks_for(counts, tasks);
  void *d_p = nullptr, *d_t = nullptr, *d_o = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  if ((r = table(c, off.data(), off.size() * sizeof(int64_t), &d_o))) return r;
  cudaError_t e = flag_launch(dtype, (const DPatch*)d_p, (const BlockTask*)d_t, (int)tasks.size(),
                              (const int64_t*)d_o, c->prm.gamma, theta, d_flags, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "flag_cells launch");
  c->launches += 1;
  return MHD_OK;
}

mhd_status mhd_ghost_fill(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, const mhd_copy* list,
                          int32_t nlist, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 0 || (n > 0 && !patches) || nlist < 0 || (nlist > 0 && !list))
    return fail(c, MHD_EINVAL, "bad arguments");
  if (nlist == 0) return MHD_OK;
  std::vector<DPatch> dp(n);
  const int dtype = n > 0 ? patches[0].dtype : 0;
  for (int p = 0; p < n; ++p) {
    if ((r = convert(c, patches[p], p, dp[p]))) return r;
    if (patches[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
  }
  std::vector<DCopy> dc(nlist);
  std::vector<int64_t> counts(nlist);
  for (int t = 0; t < nlist; ++t) {
    const mhd_copy& m = list[t];
    if (m.src < 0 || m.src >= n || m.dst < 0 || m.dst >= n)
      return fail(c, MHD_EINVAL, "copy %d: patch index out of range", t);
    const DPatch& D = dp[m.dst];
    const DPatch& S = dp[m.src];
    DCopy& o = dc[t];
    o.src = m.src;
    o.dst = m.dst;
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.box.lo[a] - D.glo[a], hi = m.box.hi[a] - D.glo[a];
      if (hi < lo || lo < -1 || hi > D.N[a])
        return fail(c, MHD_EINVAL, "copy %d: box outside the destination's arrays grown by one along axis %d", t, a);
      // source cells (and the upper face of the last one) must lie in src's interior
      const int slo = m.box.lo[a] + m.offset[a] - S.glo[a], shi = m.box.hi[a] + m.offset[a] - S.glo[a];
      if (slo < S.g || shi > S.g + S.n[a] - 1)
        return fail(c, MHD_EINVAL, "copy %d: source outside the source interior along axis %d", t, a);
      o.lo[a] = lo;
      o.ext[a] = hi - lo + 1;
      o.off[a] = (m.box.lo[a] + m.offset[a] - S.glo[a]) - lo;
      cnt *= o.ext[a];
    }
    counts[t] = cnt;
  }
  // Bottom-layer rectangles: where copy u's top layer along a lies directly
  // below copy t's bottom layer (same destination), the faces between them
  // take u's values and t skips them over the transverse extent they share.
  std::vector<std::vector<int32_t>> by_dst(n);
  for (int t = 0; t < nlist; ++t) by_dst[dc[t].dst].push_back(t);
  std::vector<DExcl> ex;
  for (int t = 0; t < nlist; ++t) {
    DCopy& o = dc[t];
    o.xr = (int32_t)ex.size();
    for (int32_t u : by_dst[o.dst]) {
      if (u == t) continue;
      const DCopy& A = dc[u];
      for (int a = 0; a < 3; ++a) {
        if (A.lo[a] + A.ext[a] != o.lo[a]) continue;
        DExcl x{};
        x.axis = a;
        bool meet = true;
        for (int k = 0, e = 0; e < 3; ++e) {
          if (e == a) continue;
          x.lo[k] = std::max(A.lo[e], o.lo[e]);
          x.hi[k] = std::min(A.lo[e] + A.ext[e], o.lo[e] + o.ext[e]) - 1;
          if (x.lo[k] > x.hi[k]) meet = false;
          ++k;
        }
        if (meet) ex.push_back(x);
      }
    }
    o.nx = (int32_t)ex.size() - o.xr;
  }
  if (ex.empty()) ex.push_back(DExcl{});  // a valid table address
  // warp tasks: groups of rows of each copy (lanes along x, see GhostTask)
  std::vector<GhostTask> tasks;
  const int gr = ghost_rows(dtype);
  for (int t = 0; t < nlist; ++t) {
    const DCopy& o = dc[t];
    if ((int64_t)o.ext[1] * o.ext[2] >= (1 << 24))
      return fail(c, MHD_EINVAL, "copy %d: more than 2^24 - 1 rows in one box", t);
    const int W = std::min(o.ext[0], 32), rows = o.ext[1] * o.ext[2], step = gr * (32 / W);
    for (int x0 = 0; x0 < o.ext[0]; x0 += 32)
      for (int r0 = 0; r0 < rows; r0 += step) tasks.push_back(GhostTask{t, r0, x0, 0});
  }
  if (tasks.size() > 0x7fffffff / kThreads) return fail(c, MHD_EINVAL, "launch too large");
  void *d_p = nullptr, *d_c = nullptr, *d_x = nullptr, *d_t = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, dc.data(), dc.size() * sizeof(DCopy), &d_c))) return r;
  if ((r = table(c, ex.data(), ex.size() * sizeof(DExcl), &d_x))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(GhostTask), &d_t))) return r;
  cudaError_t e = ghost_fill2_launch(dtype, (const DPatch*)d_p, (const DCopy*)d_c, (const DExcl*)d_x,
                                     (const GhostTask*)d_t, (int)tasks.size(), timer_of(c), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "ghost fill launch");
  c->launches += 1;
  return MHD_OK;
}

mhd_status mhd_conservation_sums(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, double* d_out8,
                                 void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 1 || !patches || !d_out8) return fail(c, MHD_EINVAL, "bad arguments");
  std::vector<DPatch> dp(n);
  std::vector<int64_t> counts(n);
  const int dtype = patches[0].dtype;
  for (int p = 0; p < n; ++p) {
    if ((r = convert(c, patches[p], p, dp[p]))) return r;
    if (patches[p].dtype != dtype) return fail(c, MHD_EINVAL, "patches of one call must share a dtype");
    counts[p] = (int64_t)dp[p].n[0] * dp[p].n[1] * dp[p].n[2];
  }
  std::vector<BlockTask> tasks;
  tasks_for(counts, tasks);
  if ((r = ensure_partials(c, tasks.size()))) return r;
  void *d_p = nullptr, *d_t = nullptr;
  if ((r = table(c, dp.data(), dp.size() * sizeof(DPatch), &d_p))) return r;
  if ((r = table(c, tasks.data(), tasks.size() * sizeof(BlockTask), &d_t))) return r;
  cudaError_t e = sums_launch(dtype, (const DPatch*)d_p, (const BlockTask*)d_t, (int)tasks.size(),
                              c->partials, d_out8, timer_of(c), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "sums launch");
  c->launches += 2;
  return MHD_OK;
}

mhd_status mhd_prolong(mhd_ctx* c, const mhd_patch_desc* coarse, int32_t nc, const mhd_patch_desc* fine,
                       int32_t nf, const mhd_prolong_item* items, int32_t n, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 0 || (n > 0 && !items)) return fail(c, MHD_EINVAL, "bad item list");
  if (n == 0) return MHD_OK;
  int dtype = -1;
  std::vector<DPatch> dc, df;
  if ((r = convert_all(c, coarse, nc, dc, &dtype))) return r;
  if ((r = convert_all(c, fine, nf, df, &dtype))) return r;
  std::vector<DBoxItem> di(n);
  std::vector<int64_t> counts(n);
  for (int t = 0; t < n; ++t) {
    const mhd_prolong_item& m = items[t];
    if (m.coarse < 0 || m.coarse >= nc || m.fine < 0 || m.fine >= nf)
      return fail(c, MHD_EINVAL, "prolong item %d: patch index out of range", t);
    const DPatch& C = dc[m.coarse];
    const DPatch& F = df[m.fine];
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.box.lo[a], hi = m.box.hi[a];
      // coarse cells and their one-cell stencil inside the coarse arrays
      if (hi < lo || lo - C.glo[a] < 1 || hi - C.glo[a] > C.N[a] - 2)
        return fail(c, MHD_EINVAL, "prolong item %d: coarse box or its stencil outside the coarse arrays", t);
      // the fine cells inside the fine arrays
      if (2 * lo - F.glo[a] < 0 || 2 * hi + 1 - F.glo[a] > F.N[a] - 1)
        return fail(c, MHD_EINVAL, "prolong item %d: fine cells outside the fine arrays", t);
      di[t].lo[a] = lo;
      di[t].ext[a] = hi - lo + 1;
      cnt *= hi - lo + 1;
    }
    di[t].a = m.coarse;
    di[t].b = m.fine;
    counts[t] = cnt;
  }
  PackedTasks pk{};
  if ((r = packed_table(c, counts, true, pk))) return r;
  void *d_c = nullptr, *d_f = nullptr, *d_i = nullptr;
  if ((r = table(c, dc.data(), dc.size() * sizeof(DPatch), &d_c))) return r;
  if ((r = table(c, df.data(), df.size() * sizeof(DPatch), &d_f))) return r;
  if ((r = table(c, di.data(), di.size() * sizeof(DBoxItem), &d_i))) return r;
  cudaError_t e = prolong_launch(dtype, (const DPatch*)d_c, (const DPatch*)d_f, (const DBoxItem*)d_i, pk,
                                 timer_of(c), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "prolong launch");
  c->launches += 1;
  return MHD_OK;
}

mhd_status mhd_restrict(mhd_ctx* c, const mhd_patch_desc* fine, int32_t nf, const mhd_patch_desc* coarse,
                        int32_t nc, const mhd_restrict_item* items, int32_t n, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 0 || (n > 0 && !items)) return fail(c, MHD_EINVAL, "bad item list");
  if (n == 0) return MHD_OK;
  int dtype = -1;
  std::vector<DPatch> dc, df;
  if ((r = convert_all(c, fine, nf, df, &dtype))) return r;
  if ((r = convert_all(c, coarse, nc, dc, &dtype))) return r;
  std::vector<DBoxItem> di(n);
  std::vector<int64_t> counts(n);
  for (int t = 0; t < n; ++t) {
    const mhd_restrict_item& m = items[t];
    if (m.coarse < 0 || m.coarse >= nc || m.fine < 0 || m.fine >= nf)
      return fail(c, MHD_EINVAL, "restrict item %d: patch index out of range", t);
    const DPatch& C = dc[m.coarse];
    const DPatch& F = df[m.fine];
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.box.lo[a], hi = m.box.hi[a];
      const int flo = F.glo[a] + F.g, fhi = flo + F.n[a] - 1;
      const int clo = C.glo[a] + C.g, chi = clo + C.n[a] - 1;
      if (hi < lo || 2 * lo < flo || 2 * hi + 1 > fhi || lo < clo - 1 || hi > chi + 1)
        return fail(c, MHD_EINVAL, "restrict item %d: box not inside the coarsened fine interior and the "
                                   "coarse interior grown by one", t);
      di[t].lo[a] = lo;
      di[t].ext[a] = hi - lo + 1;
      cnt *= hi - lo + 1;
    }
    di[t].a = m.fine;
    di[t].b = m.coarse;
    counts[t] = cnt;
  }
  std::vector<std::array<int32_t, 3>> ext(n);
  for (int t = 0; t < n; ++t)
    for (int a = 0; a < 3; ++a) ext[t][a] = di[t].ext[a];
  PackedTasks p0{}, p1{};
  if ((r = packed_table(c, counts, true, p0))) return r;
  if ((r = packed_table(c, top_counts(ext), true, p1))) return r;
  void *d_c = nullptr, *d_f = nullptr, *d_i = nullptr;
  if ((r = table(c, dc.data(), dc.size() * sizeof(DPatch), &d_c))) return r;
  if ((r = table(c, df.data(), df.size() * sizeof(DPatch), &d_f))) return r;
  if ((r = table(c, di.data(), di.size() * sizeof(DBoxItem), &d_i))) return r;
  cudaError_t e = restrict_launch(dtype, (const DPatch*)d_f, (const DPatch*)d_c, (const DBoxItem*)d_i, p0, p1,
                                  timer_of(c), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "restrict launch");
  c->launches += 2;
  return MHD_OK;
}

mhd_status mhd_restrict_prolong(mhd_ctx* c, int32_t mode, const mhd_patch_desc* fine, int32_t nf,
                                const mhd_patch_desc* coarse, int32_t nc, const mhd_level_item* items, int32_t n,
                                void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (mode != MHD_PROLONG && mode != MHD_RESTRICT) return fail(c, MHD_EINVAL, "mode %d", mode);
  if (n < 0 || (n > 0 && !items)) return fail(c, MHD_EINVAL, "bad item list");
  if (mode == MHD_PROLONG) {
    std::vector<mhd_prolong_item> it(n);
    for (int t = 0; t < n; ++t) {
      it[t].coarse = items[t].coarse;
      it[t].fine = items[t].fine;
      it[t].box = items[t].box;
    }
    return mhd_prolong(c, coarse, nc, fine, nf, it.data(), n, stream);
  }
  std::vector<mhd_restrict_item> it(n);
  for (int t = 0; t < n; ++t) {
    it[t].fine = items[t].fine;
    it[t].coarse = items[t].coarse;
    it[t].box = items[t].box;
  }
  return mhd_restrict(c, fine, nf, coarse, nc, it.data(), n, stream);
}

mhd_status mhd_reflux(mhd_ctx* c, const mhd_patch_desc* coarse, int32_t nc, double* const* corr,
                      const mhd_deposit* deps, int32_t nd, void* stream) {
  mhd_status r = begin(c);
  if (r) return r;
  if (nc < 1 || !corr || nd < 0 || (nd > 0 && !deps)) return fail(c, MHD_EINVAL, "bad arguments");
  int dtype = -1;
  std::vector<DPatch> dc;
  if ((r = convert_all(c, coarse, nc, dc, &dtype))) return r;
  // element flags of the corrected patches: one byte per element in a buffer
  // of the context that stays zero between calls (each call clears what its
  // deposits set), so no call has to clear whole patches
  std::vector<int64_t> flag_off(nc, -1);
  int64_t flag_bytes = 0;
  std::vector<DCorr> cr;
  std::vector<int> corr_idx(nc, -1);
  for (int p = 0; p < nc; ++p) {
    if (!corr[p]) continue;
    flag_off[p] = flag_bytes;
    flag_bytes += (dc[p].nelem + 15) / 16 * 16;
  }
  if ((size_t)flag_bytes > c->rflags_bytes) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "reflux flags resize");
    if (c->rflags) cudaFree(c->rflags);
    c->rflags = nullptr;
    c->rflags_bytes = 0;
    e = cudaMalloc(&c->rflags, (size_t)flag_bytes);
    if (e != cudaSuccess) return fail(c, MHD_ENOMEM, "reflux flags of %lld bytes: %s", (long long)flag_bytes,
                                      cudaGetErrorString(e));
    e = cudaMemset(c->rflags, 0, (size_t)flag_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "reflux flags clear");
    c->rflags_bytes = (size_t)flag_bytes;
  }
  unsigned char* flags = (unsigned char*)c->rflags;
  for (int p = 0; p < nc; ++p) {
    if (!corr[p]) continue;
    DCorr k;
    k.patch = p;
    k.pad = 0;
    k.count = 18 * dc[p].nelem;
    k.base = corr[p];
    k.flags = flags + flag_off[p];
    corr_idx[p] = (int)cr.size();
    cr.push_back(k);
  }
  std::vector<DDeposit> dd(nd);
  std::vector<int64_t> dcount(nd);
  int64_t marks = 0;
  for (int t = 0; t < nd; ++t) {
    const mhd_deposit& m = deps[t];
    if (m.coarse < 0 || m.coarse >= nc || !corr[m.coarse] || (m.kind != 0 && m.kind != 1) || m.axis < 0 ||
        m.axis > 2 || !m.fine || !m.coarse_reg || (m.mode != MHD_REFLUX && m.mode != MHD_SYNC))
      return fail(c, MHD_EINVAL, "deposit %d: bad coarse patch, kind, axis, mode or register", t);
    const DPatch& C = dc[m.coarse];
    DDeposit& o = dd[t];
    o.coarse = m.coarse;
    o.kind = m.kind;
    o.axis = m.axis;
    o.mode = m.mode;
    o.fine = m.fine;
    o.creg = m.coarse_reg;
    o.corr = corr[m.coarse];
    o.flags = (unsigned int*)(flags + flag_off[m.coarse]);
    o.corr_idx = corr_idx[m.coarse];
    o.pad2 = 0;
    int64_t cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int lo = m.box.lo[a], hi = m.box.hi[a];
      // the elements (face / edge index up to hi + 1) inside the coarse arrays
      if (hi < lo || lo - C.glo[a] < 0 || hi - C.glo[a] > C.N[a] - 1)
        return fail(c, MHD_EINVAL, "deposit %d: box outside the coarse arrays", t);
      // the fine elements read: 2 lo .. 2 hi + (1 along the sub-face / segment
      // axes) when refluxing; lo .. hi of the other patch when synchronising
      const bool sub = (m.kind == 0) ? (a != m.axis) : (a == m.axis);
      const int f0 = m.mode == MHD_SYNC ? lo : 2 * lo, f1 = m.mode == MHD_SYNC ? hi : 2 * hi + (sub ? 1 : 0);
      if (f0 < m.fine_box.lo[a] || f1 > m.fine_box.hi[a])
        return fail(c, MHD_EINVAL, "deposit %d: fine register box does not hold the fine elements", t);
      o.lo[a] = lo;
      o.ext[a] = hi - lo + 1;
      o.flo[a] = m.fine_box.lo[a];
      o.fext[a] = m.fine_box.hi[a] - m.fine_box.lo[a] + 1;
      cnt *= o.ext[a];
    }
    dcount[t] = cnt;
    // elements one deposit element can flag: 2 for a face, 4 for an edge
    marks += cnt * (m.kind == 0 ? 2 : 4);
  }
  std::vector<BlockTask> td;
  tasks_for(dcount, td);
  // the list of flagged elements (and its count) in the arena
  if ((r = ensure_scratch(c, (size_t)(marks + 1) * 8))) return r;
  RefluxList L;
  L.count = (unsigned long long*)c->scratch;
  L.entries = L.count + 1;
  L.capacity = (unsigned long long)marks;
  void *d_c = nullptr, *d_r = nullptr, *d_d = nullptr, *d_td = nullptr;
  if ((r = table(c, dc.data(), dc.size() * sizeof(DPatch), &d_c))) return r;
  if ((r = table(c, cr.data(), cr.size() * sizeof(DCorr), &d_r))) return r;
  if ((r = table(c, dd.data(), dd.size() * sizeof(DDeposit), &d_d))) return r;
  if ((r = table(c, td.data(), td.size() * sizeof(BlockTask), &d_td))) return r;
  cudaError_t e = reflux_launch(dtype, (const DPatch*)d_c, (const DCorr*)d_r, L, (const DDeposit*)d_d,
                                (const BlockTask*)d_td, (int)td.size(), timer_of(c), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "reflux launch");
  if (nd > 0) c->launches += 3;
  return MHD_OK;
}


// ---------------------------------------------------------------- flux registers
}  // extern "C"

struct mhd_fluxreg {
  int device = 0;
  double* base = nullptr;
  size_t count = 0;
  struct Item {
    int64_t off;
    mhd_box box;
  };
  std::vector<Item> faces;  // patch * 6 + 2 * axis + side
  std::vector<Item> edges;  // patch * 12 + 2 * (2 * face axis + side) + (edge axis == face axis + 1 (mod 3) ? 0 : 1)
};

extern "C" {

mhd_status mhd_fluxreg_create(mhd_ctx* c, const mhd_patch_desc* patches, int32_t n, mhd_fluxreg** out) {
  if (!out) return MHD_EINVAL;
  *out = nullptr;
  mhd_status r = begin(c);
  if (r) return r;
  if (n < 1 || !patches) return fail(c, MHD_EINVAL, "fluxreg: bad arguments");
  std::unique_ptr<mhd_fluxreg> g(new mhd_fluxreg);
  g->device = c->device;
  int64_t off = 0;
  for (int p = 0; p < n; ++p) {
    const mhd_box& in = patches[p].interior;
    int64_t len[3];
    for (int a = 0; a < 3; ++a) {
      len[a] = (int64_t)in.hi[a] - in.lo[a] + 1;
      if (len[a] < 1) return fail(c, MHD_EINVAL, "fluxreg: patch %d has an empty interior", p);
    }
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        mhd_fluxreg::Item it;
        it.box = in;
        it.box.lo[d] = it.box.hi[d] = side ? in.hi[d] + 1 : in.lo[d];
        it.off = off;
        g->faces.push_back(it);
        off += 5 * (len[0] * len[1] * len[2] / len[d]);
      }
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side)
        for (int k = 0; k < 2; ++k) {
          const int a = (d + 1 + k) % 3, t = (d + 2 - k) % 3;  // edge axis, remaining transverse axis
          mhd_fluxreg::Item it;
          it.box = in;
          it.box.lo[d] = it.box.hi[d] = side ? in.hi[d] + 1 : in.lo[d];
          it.box.hi[t] = in.hi[t] + 1;
          it.off = off;
          g->edges.push_back(it);
          off += len[a] * (len[t] + 1);
        }
  }
  g->count = (size_t)off;
  cudaError_t e = cudaMalloc(&g->base, g->count * sizeof(double));
  if (e != cudaSuccess) return fail(c, MHD_ENOMEM, "fluxreg: %zu doubles: %s", g->count, cudaGetErrorString(e));
  e = cudaMemset(g->base, 0, g->count * sizeof(double));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(g->base);
    return cuda_fail(c, e, "fluxreg: zero");
  }
  *out = g.release();
  return MHD_OK;
}

void mhd_fluxreg_destroy(mhd_fluxreg* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  if (g->base) cudaFree(g->base);
  delete g;
}

double* mhd_fluxreg_face(const mhd_fluxreg* g, int32_t patch, int32_t axis, int32_t side, mhd_box* box) {
  if (!g || patch < 0 || axis < 0 || axis > 2 || side < 0 || side > 1) return nullptr;
  const size_t k = (size_t)patch * 6 + 2 * axis + side;
  if (k >= g->faces.size()) return nullptr;
  if (box) *box = g->faces[k].box;
  return g->base + g->faces[k].off;
}

double* mhd_fluxreg_edge(const mhd_fluxreg* g, int32_t patch, int32_t face_axis, int32_t side, int32_t edge_axis,
                         mhd_box* box) {
  if (!g || patch < 0 || face_axis < 0 || face_axis > 2 || side < 0 || side > 1 || edge_axis < 0 ||
      edge_axis > 2 || edge_axis == face_axis)
    return nullptr;
  const int k = edge_axis == (face_axis + 1) % 3 ? 0 : 1;
  const size_t i = (size_t)patch * 12 + 2 * (2 * face_axis + side) + k;
  if (i >= g->edges.size()) return nullptr;
  if (box) *box = g->edges[i].box;
  return g->base + g->edges[i].off;
}

mhd_status mhd_fluxreg_zero(mhd_fluxreg* g, void* stream) {
  if (!g) return MHD_EINVAL;
  if (cudaSetDevice(g->device) != cudaSuccess) return MHD_ECUDA;
  return cudaMemsetAsync(g->base, 0, g->count * sizeof(double), (cudaStream_t)stream) == cudaSuccess ? MHD_OK
                                                                                                       : MHD_ECUDA;
}

}  // extern "C"
