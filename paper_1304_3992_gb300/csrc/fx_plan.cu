// fx_plan.cu -- plans: the batched persistent kernels over a tile queue (CUDA
// graph replay), the per-batch unit height and the tuner, the device status
// word, and the end-to-end entry points on host buffers (a copy / kernel /
// copy pipeline over row chunks of one or many images).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "fx_internal.h"
#include "fx_plan_kernels.cuh"
#include "fx_stream.cuh"
#include "fx_tile.cuh"

namespace fx {
namespace {

__global__ void __launch_bounds__(256) batch_kernel_general(const unsigned char *table,
                                                            unsigned long long *counter, int *status,
                                                            const __grid_constant__ KParams kp8,
                                                            const __grid_constant__ KParams kp16) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_unit;
  const BatchHeader *hdr = reinterpret_cast<const BatchHeader *>(table);
  const BatchImage *ims = reinterpret_cast<const BatchImage *>(table + sizeof(BatchHeader));
  const long long total = hdr->total_units;
  for (;;) {
    if (threadIdx.x == 0) s_unit = static_cast<long long>(atomicAdd(counter, 1ULL));
    __syncthreads();
    const long long u = s_unit;
    __syncthreads();
    if (u >= total) break;
    const BatchImage &b = ims[find_image(ims, hdr->n, u)];
    if (b.units_x <= 0 || (b.elem != 1 && b.elem != 2)) {
      if (threadIdx.x == 0) atomicOr(status, kStatusBadDescriptor);
      continue;
    }
    const ImageView v = view_of(b);
    const long long local = u - b.unit_begin;
    const int64_t ux = local % b.units_x, uy = local / b.units_x;
    if (b.elem == 1) gen::general_tile<uint8_t>(v, kp8, ux * gen::TW, uy * gen::TH, smem);
    else gen::general_tile<uint16_t>(v, kp16, ux * gen::TW, uy * gen::TH, smem);
    __syncthreads();
  }
}

}  // namespace

// The narrow class's selectors (the other classes are in fx_plan_compact.cu,
// fx_plan_wide.cu and fx_plan_xwide.cu).
const void *plan_fast_kernel_narrow(const KParams &kp, int g) { return fast_kernel_of<kNarrowRm>(kp, g); }
const void *plan_redo_kernel_narrow(const KParams &kp) { return redo_kernel_of<kNarrowRm>(kp); }
const void *plan_fast_kernel_compact(const KParams &kp, int g);
const void *plan_redo_kernel_compact(const KParams &kp);
const void *plan_fast_kernel_wide(const KParams &kp, int g);
const void *plan_redo_kernel_wide(const KParams &kp);
const void *plan_fast_kernel_xwide(const KParams &kp, int g);
const void *plan_redo_kernel_xwide(const KParams &kp);

const void *plan_fast_kernel(int rm_class, const KParams &kp, int g) {
  if (rm_class == kCompactRm) return plan_fast_kernel_compact(kp, g);
  if (rm_class == kWideRm) return plan_fast_kernel_wide(kp, g);
  if (rm_class == kXWideRm) return plan_fast_kernel_xwide(kp, g);
  return plan_fast_kernel_narrow(kp, g);
}
const void *plan_redo_kernel(int rm_class, const KParams &kp) {
  if (rm_class == kCompactRm) return plan_redo_kernel_compact(kp);
  if (rm_class == kWideRm) return plan_redo_kernel_wide(kp);
  if (rm_class == kXWideRm) return plan_redo_kernel_xwide(kp);
  return plan_redo_kernel_narrow(kp);
}

}  // namespace fx

using namespace fx;

// Staging slots of the host-buffer path: copy-in, kernel and copy-out of three
// consecutive row chunks run at the same time.
constexpr int kHostSlots = 3;

struct fx_plan {
  fx_params params;
  KParams kp8, kp16;
  fx_status st16;  // FX_ERR_RANGE when 16-bit images cannot be evaluated exactly
  bool fast;
  int rm_class;  // strip class of the streaming path (kCompactRm, kNarrowRm, kWideRm or kXWideRm)
  int device, max_images, num_sms;
  // batch workspace, double-buffered: graph i copies host table i into device
  // table i and runs on queue counters i, so two replays (e.g. from two
  // streams) can be in flight; a third waits on the host for the first
  unsigned char *d_table[2];
  unsigned char *h_table[2];
  cudaEvent_t h_free[2];
  int h_next;
  unsigned long long *d_counter[2];
  int *d_status;
  cudaGraphExec_t graph[2];
  int unit_w, unit_h, ctas_per_sm;
  bool auto_h;  // pick the unit height per call (until fx_plan_set_tile fixes it)
  size_t smem;
  // end-to-end path on host buffers
  cudaStream_t s_h2d, s_comp, s_d2h;
  // host-buffer path: a ring of kHostSlots staging buffers and their events
  void *d_in[kHostSlots];
  uint8_t *d_out[kHostSlots];
  size_t in_cap, out_cap;
  cudaEvent_t ev_in[kHostSlots], ev_comp[kHostSlots], ev_out[kHostSlots];
};

namespace {

// Makes the plan's device current for one entry point and restores the
// caller's current device on return.
struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void destroy_graphs(fx_plan *p) {
  for (int i = 0; i < 2; ++i)
    if (p->graph[i]) {
      cudaGraphExecDestroy(p->graph[i]);
      p->graph[i] = nullptr;
    }
}

size_t unit_smem(const fx_plan *p) {
  if (p->fast) return fast_smem_bytes(std::max(p->kp8.r_in, p->kp16.r_in), p->unit_w, p->unit_h);
  return std::max(gen::general_smem_bytes(p->kp8), gen::general_smem_bytes(p->kp16));
}

// Graph i: copy host table i to the device, zero the queue counters, run the
// persistent kernel (general path), or the four group kernels of the streaming
// path as independent nodes (a group's CTAs take the SMs that the previous
// group's drained queue frees) followed by the redo pass.  The table copy has
// a fixed size so the graph never changes.
fx_status build_graph(fx_plan *p, int i) {
  p->smem = unit_smem(p);
  const void *fn = p->fast ? plan_fast_kernel(p->rm_class, p->kp8, 0) : reinterpret_cast<const void *>(&batch_kernel_general);
  if (!p->fast &&  // the streaming kernels use static shared memory only
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
    return FX_ERR_CUDA;
  cudaGraph_t g;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return FX_ERR_CUDA;
  cudaGraphNode_t n_copy, n_zero, n_kern;
  cudaMemcpy3DParms cp;
  std::memset(&cp, 0, sizeof cp);
  cp.srcPtr = make_cudaPitchedPtr(p->h_table[i], table_bytes(p->max_images), table_bytes(p->max_images), 1);
  cp.dstPtr = make_cudaPitchedPtr(p->d_table[i], table_bytes(p->max_images), table_bytes(p->max_images), 1);
  cp.extent = make_cudaExtent(table_bytes(p->max_images), 1, 1);
  cp.kind = cudaMemcpyHostToDevice;
  cudaMemsetParams ms;
  std::memset(&ms, 0, sizeof ms);
  ms.dst = p->d_counter[i];
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = 2 * kGroups;  // the queue counters
  ms.height = 1;
  ms.pitch = 8 * kGroups;
  const unsigned char *tab = p->d_table[i];
  unsigned long long *ctr = p->d_counter[i];
  int *stp = p->d_status;
  KParams k8 = p->kp8, k16 = p->kp16;
  void *args[] = {&tab, &ctr, &stp, &k8, &k16};
  cudaKernelNodeParams kn;
  std::memset(&kn, 0, sizeof kn);
  kn.func = const_cast<void *>(fn);
  kn.gridDim = dim3(static_cast<unsigned>(p->num_sms * p->ctas_per_sm));
  kn.blockDim = dim3(p->fast ? 32 * kWarpsPerCta : 256);
  kn.sharedMemBytes = static_cast<unsigned>(p->smem);
  kn.kernelParams = args;
  cudaError_t e = cudaGraphAddMemcpyNode(&n_copy, g, nullptr, 0, &cp);
  if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&n_zero, g, &n_copy, 1, &ms);
  if (!p->fast) {
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n_kern, g, &n_zero, 1, &kn);
  } else {
    cudaGraphNode_t n_grp[kGroups];
    for (int gi = 0; gi < kGroups && e == cudaSuccess; ++gi) {
      KParams *kg = gi % 2 == 1 ? &k8 : &k16;  // groups 1 and 3 hold the uint8 images
      void *gargs[] = {&tab, &ctr, &stp, kg};
      cudaKernelNodeParams kf = kn;
      kf.func = const_cast<void *>(plan_fast_kernel(p->rm_class, p->kp8, gi));
      // a kernel compiled for the plan's parameters, if any (fx_specialize); groups 0 / 1
      // hold the aligned-load images, 2 / 3 the others
      if (const void *jk = specialized_batch_kernel(gi % 2 == 1 ? p->kp8 : p->kp16, gi % 2 == 1 ? 1 : 2, gi < 2,
                                                    p->rm_class))
        kf.func = const_cast<void *>(jk);
      kf.kernelParams = gargs;
      e = cudaGraphAddKernelNode(&n_grp[gi], g, &n_zero, 1, &kf);
    }
    // the integer (or wide) redo pass after all groups, one wave of CTAs
    cudaKernelNodeParams kr = kn;
    kr.func = const_cast<void *>(plan_redo_kernel(p->rm_class, p->kp8));
    kr.sharedMemBytes = 0;
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kr.func, 32 * kWarpsPerCta, 0);
    kr.gridDim = dim3(static_cast<unsigned>(p->num_sms * std::max(1, occ)));
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n_kern, g, n_grp, kGroups, &kr);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->graph[i], g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? FX_OK : FX_ERR_CUDA;
}

fx_status rebuild(fx_plan *p) {
  destroy_graphs(p);
  for (int i = 0; i < 2; ++i) {
    fx_status st = build_graph(p, i);
    if (st != FX_OK) return st;
  }
  return FX_OK;
}

fx_status fill_table(fx_plan *p, unsigned char *h, const fx_image_desc *d, int32_t n) {
  BatchHeader *hdr = reinterpret_cast<BatchHeader *>(h);
  BatchImage *ims = reinterpret_cast<BatchImage *>(h + sizeof(BatchHeader));
  const int uwx = p->fast ? strip_width(p->kp8.source == 1, p->rm_class) : gen::TW;  // output columns per unit
  int uh = p->fast ? p->unit_h : gen::TH;
  if (p->fast && p->auto_h) {
    // the wave model of fx_extract over the whole batch: a warp walks uh rows
    // plus the pipeline overhead (the batched units run the whole block
    // schedule: ring prefill and three to five blocks of delay), and the batch
    // takes about ceil(units / warps) unit times
    const int64_t slots = static_cast<int64_t>(p->num_sms) * p->ctas_per_sm * kWarpsPerCta;
    const int64_t overhead = 56 + 16 * ((p->kp8.nhmf == 2 ? 1 : 0) + (p->kp8.source == 1 ? 1 : 0));
    int64_t best_cost = INT64_MAX;
    for (int h = 1024; h >= 16; h -= 16) {
      int64_t units = 0;
      for (int32_t i = 0; i < n; ++i)
        units += std::max<int64_t>(1, (d[i].width + uwx - 1) / uwx) * std::max<int64_t>(1, (d[i].height + h - 1) / h);
      const int64_t cost = (units + slots - 1) / slots * (h + overhead);
      if (cost < best_cost) {
        best_cost = cost;
        uh = h;
      }
    }
  }
  const int uw = p->fast ? p->unit_w : gen::TW;
  int64_t total = 0, group_end[kGroups] = {0, 0, 0, 0};
  // On the streaming path the queue runs through the images in four groups
  // (group_of): one aligned load per lane (uint16, then uint8), then pixel by
  // pixel (uint16, then uint8); each group is one kernel with one strip loop.
  int32_t slot = 0;
  for (int pass = 0; pass < (p->fast ? 4 : 1); ++pass)
  for (int32_t i = 0; i < n; ++i) {
    const int64_t op = d[i].out_pitch ? d[i].out_pitch : d[i].width;
    const int64_t elem = d[i].dtype == FX_U8 ? 1 : 2;
    const bool pair = p->fast && pair_loads_ok(d[i].img, d[i].width, d[i].pitch_bytes, elem);
    if (p->fast && group_of(pair, static_cast<int>(elem)) != pass) continue;
    fx_status st = check_image(d[i].img, d[i].width, d[i].height, d[i].pitch_bytes, d[i].dtype,
                               d[i].out_mask, op);
    if (st != FX_OK) return st;
    if (d[i].dtype == FX_U16 && p->st16 != FX_OK) return p->st16;
    BatchImage &b = ims[slot++];
    b.img = d[i].img;
    b.width = d[i].width;
    b.height = d[i].height;
    b.pitch = d[i].pitch_bytes;
    b.out = d[i].out_mask;
    b.out_pitch = op;
    b.elem = d[i].dtype == FX_U8 ? 1 : 2;
    b.pad = 0;
    b.units_x = (b.width + uwx - 1) / uwx;
    b.unit_begin = total;
    total += b.units_x * ((b.height + uh - 1) / uh);
    if (p->fast) group_end[pass] = total;
  }
  if (slot != n) return FX_ERR_INVALID_ARG;  // every descriptor belongs to exactly one group
  // outputs must not overlap each other (inputs were checked per descriptor)
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j = i + 1; j < n; ++j) {
      uintptr_t a0 = reinterpret_cast<uintptr_t>(ims[i].out), a1 = a0 + (ims[i].height - 1) * ims[i].out_pitch + ims[i].width;
      uintptr_t b0 = reinterpret_cast<uintptr_t>(ims[j].out), b1 = b0 + (ims[j].height - 1) * ims[j].out_pitch + ims[j].width;
      uintptr_t c0 = reinterpret_cast<uintptr_t>(ims[j].img), c1 = c0 + (ims[j].height - 1) * ims[j].pitch + ims[j].width * ims[j].elem;
      uintptr_t e0 = reinterpret_cast<uintptr_t>(ims[i].img), e1 = e0 + (ims[i].height - 1) * ims[i].pitch + ims[i].width * ims[i].elem;
      if ((a0 < b1 && b0 < a1) || (a0 < c1 && c0 < a1) || (b0 < e1 && e0 < b1)) return FX_ERR_INVALID_ARG;
    }
  hdr->total_units = total;
  for (int gi = 0; gi < kGroups; ++gi) {  // a group with no image ends where the previous one does
    if (gi > 0) group_end[gi] = std::max(group_end[gi], group_end[gi - 1]);
    hdr->group_end[gi] = p->fast ? group_end[gi] : total;
  }
  hdr->n = n;
  hdr->unit_w = uw;
  hdr->unit_h = uh;
  hdr->pad = 0;
  return FX_OK;
}

void free_host_path(fx_plan *p) {
  for (int i = 0; i < kHostSlots; ++i) {
    if (p->d_in[i]) cudaFree(p->d_in[i]);
    if (p->d_out[i]) cudaFree(p->d_out[i]);
    p->d_in[i] = nullptr;
    p->d_out[i] = nullptr;
  }
  p->in_cap = p->out_cap = 0;
}

}  // namespace

extern "C" {

fx_status fx_plan_create(fx_plan **out, const fx_params *params, int32_t max_images, int32_t device) {
  if (!out || max_images < 1 || max_images > (1 << 20)) return FX_ERR_INVALID_ARG;
  *out = nullptr;
  fx_params def;
  if (!params) {
    fx_params_default(&def, FX_U16, 0);
    params = &def;
  }
  if (params->struct_size != sizeof(fx_params)) return FX_ERR_INVALID_ARG;
  fx_plan *p = new (std::nothrow) fx_plan;
  if (!p) return FX_ERR_NOMEM;
  std::memset(static_cast<void *>(p), 0, sizeof(*p));
  p->params = *params;
  fx_status st = make_kparams(params, 255, &p->kp8);
  if (st != FX_OK) {
    delete p;
    return st;
  }
  p->st16 = make_kparams(params, 65535, &p->kp16);
  if (p->st16 != FX_OK) p->kp16 = p->kp8;
  // the streaming path for median radii up to 11 (both parameter sets share the list)
  p->fast = fast_path_supported(p->kp8) && fast_path_supported(p->kp16);
  p->rm_class = strip_class(p->kp8);
  p->device = device;
  p->max_images = max_images;
  p->unit_w = strip_width(p->kp8.source == 1, p->rm_class);
  p->unit_h = kDefaultUnitH;
  p->ctas_per_sm = p->fast ? kBatchCtas : 2;
  p->auto_h = true;
  DeviceScope dev(device);
  if (!dev.ok || cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete p;
    return FX_ERR_CUDA;
  }
  bool ok = cudaMalloc(&p->d_status, 4) == cudaSuccess && cudaMemset(p->d_status, 0, 4) == cudaSuccess;
  for (int i = 0; i < 2 && ok; ++i) {
    ok = cudaMalloc(&p->d_table[i], table_bytes(max_images)) == cudaSuccess &&
         cudaMalloc(&p->d_counter[i], 8 * kGroups) == cudaSuccess &&
         cudaMallocHost(&p->h_table[i], table_bytes(max_images)) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->h_free[i], cudaEventDisableTiming) == cudaSuccess;
    if (ok) std::memset(p->h_table[i], 0, table_bytes(max_images));
  }
  ok = ok && cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
  for (int i = 0; i < kHostSlots && ok; ++i)
    ok = cudaEventCreateWithFlags(&p->ev_in[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->ev_comp[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&p->ev_out[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok || rebuild(p) != FX_OK) {
    fx_plan_destroy(p);
    return ok ? FX_ERR_CUDA : FX_ERR_NOMEM;
  }
  *out = p;
  return FX_OK;
}

fx_status fx_plan_destroy(fx_plan *p) {
  if (!p) return FX_ERR_INVALID_ARG;
  DeviceScope dev(p->device);
  for (int i = 0; i < 2; ++i)
    if (p->h_free[i]) cudaEventSynchronize(p->h_free[i]);
  if (p->s_h2d) cudaStreamSynchronize(p->s_h2d);
  if (p->s_comp) cudaStreamSynchronize(p->s_comp);
  if (p->s_d2h) cudaStreamSynchronize(p->s_d2h);
  destroy_graphs(p);
  free_host_path(p);
  for (int i = 0; i < 2; ++i) {
    if (p->h_table[i]) cudaFreeHost(p->h_table[i]);
    if (p->h_free[i]) cudaEventDestroy(p->h_free[i]);
  }
  for (int i = 0; i < kHostSlots; ++i) {
    if (p->ev_in[i]) cudaEventDestroy(p->ev_in[i]);
    if (p->ev_comp[i]) cudaEventDestroy(p->ev_comp[i]);
    if (p->ev_out[i]) cudaEventDestroy(p->ev_out[i]);
  }
  for (int i = 0; i < 2; ++i) {
    if (p->d_table[i]) cudaFree(p->d_table[i]);
    if (p->d_counter[i]) cudaFree(p->d_counter[i]);
  }
  if (p->d_status) cudaFree(p->d_status);
  if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
  if (p->s_comp) cudaStreamDestroy(p->s_comp);
  if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
  delete p;
  return FX_OK;
}

fx_status fx_extract_batch(fx_plan *p, const fx_image_desc *descs, int32_t n, void *stream) {
  NvtxRange range("fx_extract_batch");
  if (!p || !descs || n < 1 || n > p->max_images) return FX_ERR_INVALID_ARG;
  DeviceScope dev(p->device);
  if (!dev.ok) return FX_ERR_CUDA;
  const int i = p->h_next;
  // the previous replay that read host table i must have copied it out
  if (cudaEventSynchronize(p->h_free[i]) != cudaSuccess) return FX_ERR_CUDA;
  fx_status st = fill_table(p, p->h_table[i], descs, n);
  if (st != FX_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaGraphLaunch(p->graph[i], s) != cudaSuccess) return FX_ERR_CUDA;
  if (cudaEventRecord(p->h_free[i], s) != cudaSuccess) return FX_ERR_CUDA;
  p->h_next = i ^ 1;
  return FX_OK;
}

fx_status fx_plan_set_tile(fx_plan *p, int32_t tile_w, int32_t tile_h, int32_t ctas_per_sm) {
  if (!p || ctas_per_sm < 1 || ctas_per_sm > kMaxCtasPerSm) return FX_ERR_INVALID_ARG;
  // tile_h 0: the height is picked per batch (the wave model in fill_table)
  const bool automatic = tile_h == 0;
  const int th = automatic ? kDefaultUnitH : tile_h;
  if (tile_w != strip_width(p->kp8.source == 1, p->rm_class) || th < 16 || th > 8192 || th % 16 != 0)
    return FX_ERR_INVALID_ARG;
  DeviceScope dev(p->device);
  if (!dev.ok) return FX_ERR_CUDA;
  for (int i = 0; i < 2; ++i)
    if (cudaEventSynchronize(p->h_free[i]) != cudaSuccess) return FX_ERR_CUDA;
  p->unit_w = tile_w;
  p->unit_h = automatic ? kDefaultUnitH : tile_h;
  p->ctas_per_sm = ctas_per_sm;
  p->auto_h = automatic;
  return rebuild(p);
}

fx_status fx_plan_autotune(fx_plan *p, const fx_image_desc *descs, int32_t n, void *stream,
                           int32_t *tile_w, int32_t *tile_h, int32_t *ctas_per_sm) {
  NvtxRange range("fx_plan_autotune");
  if (!p || !descs || n < 1 || n > p->max_images) return FX_ERR_INVALID_ARG;
  DeviceScope dev(p->device);
  if (!dev.ok) return FX_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FX_ERR_CUDA;
  float best = 1e30f;
  int bw = p->unit_w, bh = p->unit_h, bc = p->ctas_per_sm;
  fx_status st = FX_OK;
  // candidates: the automatic height (0), then the fixed heights
  for (int c = -1; c < kNumUnitHeights && st == FX_OK; ++c) {
    const int uw = strip_width(p->kp8.source == 1, p->rm_class), uh = c < 0 ? 0 : kUnitHeights[c];
    // CTAs per SM: the streaming kernels' default and two and four fewer, the
    // general kernel's 1 .. 8 (its occupancy decides)
    const int cands_fast[3] = {kBatchCtas, std::max(1, kBatchCtas - 2), std::max(1, kBatchCtas - 4)};
    for (int ci = 0; ci < (p->fast ? 3 : 8) && st == FX_OK; ++ci) {
      const int cps = p->fast ? cands_fast[ci] : ci + 1;
      if (!p->fast && uh != 0) continue;
      if ((st = fx_plan_set_tile(p, uw, uh, cps)) != FX_OK) break;
      int occ = 0;
      if (p->fast) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, plan_fast_kernel(p->rm_class, p->kp8, 0), 32 * kWarpsPerCta, 0);
      else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel_general, 256, p->smem);
      if (occ < cps) continue;
      float t_best = 1e30f;
      for (int rep = 0; rep < 4 && st == FX_OK; ++rep) {
        cudaEventRecord(e0, s);
        st = fx_extract_batch(p, descs, n, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = FX_ERR_CUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t_best = std::min(t_best, ms);
      }
      if (t_best < best) {
        best = t_best;
        bw = uw;
        bh = uh;
        bc = cps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FX_OK) return st;
  st = fx_plan_set_tile(p, bw, bh, bc);
  if (tile_w) *tile_w = bw;
  if (tile_h) *tile_h = bh;
  if (ctas_per_sm) *ctas_per_sm = bc;
  return st;
}

fx_status fx_get_device_status(fx_plan *p, void *stream) {
  if (!p) return FX_ERR_INVALID_ARG;
  DeviceScope dev(p->device);
  if (!dev.ok) return FX_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  if (cudaMemcpyAsync(&h, p->d_status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemsetAsync(p->d_status, 0, 4, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return FX_ERR_CUDA;
  return h == 0 ? FX_OK : FX_ERR_INVALID_ARG;
}

}  // extern "C"

namespace {

// Host buffers in, host mask out.  Images go to the device in row chunks;
// chunk k+1's upload overlaps chunk k's kernel and chunk k-1's download, across
// image boundaries.  Each chunk carries the input halo rows its outputs need,
// so results equal fx_extract's.
struct HostJob {  // one image of the host-buffer path
  const unsigned char *src;
  int64_t width, height, pitch, elem;
  uint8_t *dst;
  int64_t out_pitch;
};

// Rows per chunk: about 64 MiB of input (enough strips to fill the GPU, small
// enough that copies and kernels of neighbouring chunks overlap), >= 64 rows.
int64_t chunk_rows(const HostJob &j) {
  const int64_t dpitch = (j.width * j.elem + 255) / 256 * 256;
  return std::min(j.height, std::max<int64_t>(64, (64LL << 20) / dpitch));
}

// All chunks of all images through the slot ring: the copy-in of a chunk, the
// kernel of the one before and the copy-out of the one before that overlap.
fx_status host_pipeline(fx_plan *p, const HostJob *jobs, int32_t n) {
  NvtxRange range("fx host pipeline");
  DeviceScope dev(p->device);
  if (!dev.ok) return FX_ERR_CUDA;
  size_t need_in = 0, need_out = 0;
  for (int32_t i = 0; i < n; ++i) {
    const KParams &kp = jobs[i].elem == 1 ? p->kp8 : p->kp16;
    const int64_t dpitch = (jobs[i].width * jobs[i].elem + 255) / 256 * 256, band = chunk_rows(jobs[i]);
    need_in = std::max(need_in, static_cast<size_t>(std::min(jobs[i].height, band + 2 * kp.r_in) * dpitch));
    need_out = std::max(need_out, static_cast<size_t>(band * jobs[i].width));
  }
  if (need_in > p->in_cap || need_out > p->out_cap) {
    cudaStreamSynchronize(p->s_h2d);
    cudaStreamSynchronize(p->s_comp);
    cudaStreamSynchronize(p->s_d2h);
    free_host_path(p);
    for (int i = 0; i < kHostSlots; ++i)
      if (cudaMalloc(&p->d_in[i], need_in) != cudaSuccess || cudaMalloc(&p->d_out[i], need_out) != cudaSuccess) {
        free_host_path(p);
        return FX_ERR_NOMEM;
      }
    p->in_cap = need_in;
    p->out_cap = need_out;
  }
  cudaError_t e = cudaSuccess;
  int k = 0;
  for (int32_t i = 0; i < n && e == cudaSuccess; ++i) {
    const HostJob &jb = jobs[i];
    const KParams &kp = jb.elem == 1 ? p->kp8 : p->kp16;
    const int64_t r = kp.r_in, width = jb.width, height = jb.height, elem = jb.elem;
    const int64_t dpitch = (width * elem + 255) / 256 * 256, band = chunk_rows(jb);
    // the call's first and last chunks are a quarter of the others: the
    // pipeline starts and drains sooner (+1.3 % on four 16384^2 bands)
    const int64_t small = std::max<int64_t>(64, band / 4);
    for (int64_t y0 = 0, y1 = 0; y0 < height && e == cudaSuccess; y0 = y1, ++k) {
      const int slot = k % kHostSlots;
      NvtxRange chunk_range("fx host chunk (copy in, extract, copy out)");
      int64_t rows = band;
      if (i == 0 && y0 == 0) rows = small;
      const int64_t left = height - y0;
      if (i == n - 1 && left > small && left <= band + small) rows = left - small;
      y1 = std::min(height, y0 + rows);
      const int64_t a = std::max<int64_t>(0, y0 - r), b = std::min(height, y1 + r);
      // slot reuse: the kernel kHostSlots chunks ago must be done reading
      // d_in[slot], and its copy-out done reading d_out[slot]
      e = cudaStreamWaitEvent(p->s_h2d, p->ev_comp[slot], 0);
      if (e == cudaSuccess) {
        if (jb.pitch == dpitch)  // contiguous rows: one linear copy
          e = cudaMemcpyAsync(p->d_in[slot], jb.src + a * jb.pitch, (b - a) * dpitch, cudaMemcpyHostToDevice,
                              p->s_h2d);
        else
          e = cudaMemcpy2DAsync(p->d_in[slot], dpitch, jb.src + a * jb.pitch, jb.pitch, width * elem, b - a,
                                cudaMemcpyHostToDevice, p->s_h2d);
      }
      if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[slot], p->s_h2d);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_comp, p->ev_in[slot], 0);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_comp, p->ev_out[slot], 0);
      if (e == cudaSuccess) {
        ImageView v{p->d_in[slot], width, height, dpitch, a, static_cast<int32_t>(elem), p->d_out[slot], width,
                    y0, y1, b};
        e = launch_extract(v, kp, p->s_comp);
      }
      if (e == cudaSuccess) e = cudaEventRecord(p->ev_comp[slot], p->s_comp);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_d2h, p->ev_comp[slot], 0);
      if (e == cudaSuccess) {
        if (jb.out_pitch == width)
          e = cudaMemcpyAsync(jb.dst + y0 * jb.out_pitch, p->d_out[slot], (y1 - y0) * width, cudaMemcpyDeviceToHost,
                              p->s_d2h);
        else
          e = cudaMemcpy2DAsync(jb.dst + y0 * jb.out_pitch, jb.out_pitch, p->d_out[slot], width, width, y1 - y0,
                                cudaMemcpyDeviceToHost, p->s_d2h);
      }
      if (e == cudaSuccess) e = cudaEventRecord(p->ev_out[slot], p->s_d2h);
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(p->s_d2h);
  cudaStreamSynchronize(p->s_comp);
  cudaStreamSynchronize(p->s_h2d);
  return (e == cudaSuccess && e2 == cudaSuccess) ? FX_OK : FX_ERR_CUDA;
}

fx_status host_job(fx_plan *p, const void *img_host, int64_t width, int64_t height, int64_t pitch_bytes,
                   int32_t dtype, uint8_t *out_host, int64_t out_pitch, HostJob *j) {
  if (!img_host || !out_host) return FX_ERR_INVALID_ARG;
  if (dtype != FX_U8 && dtype != FX_U16) return FX_ERR_INVALID_ARG;
  const int64_t elem = dtype == FX_U8 ? 1 : 2;
  if (out_pitch == 0) out_pitch = width;
  if (width < 1 || height < 1 || width > (1LL << 30) || height > (1LL << 30) || pitch_bytes < width * elem ||
      pitch_bytes % elem || pitch_bytes > 0xFFFFFFFFLL || out_pitch < width || out_pitch > 0xFFFFFFFFLL)
    return FX_ERR_INVALID_ARG;
  if (dtype == FX_U16 && p->st16 != FX_OK) return p->st16;
  *j = HostJob{static_cast<const unsigned char *>(img_host), width, height, pitch_bytes, elem, out_host, out_pitch};
  return FX_OK;
}

}  // namespace

extern "C" {

fx_status fx_extract_host(fx_plan *p, const void *img_host, int64_t width, int64_t height,
                          int64_t pitch_bytes, fx_dtype dtype, uint8_t *out_host, int64_t out_pitch) {
  if (!p) return FX_ERR_INVALID_ARG;
  HostJob j;
  fx_status st = host_job(p, img_host, width, height, pitch_bytes, dtype, out_host, out_pitch, &j);
  return st != FX_OK ? st : host_pipeline(p, &j, 1);
}

fx_status fx_extract_host_batch(fx_plan *p, const fx_image_desc *descs, int32_t n) {
  if (!p || !descs || n < 1) return FX_ERR_INVALID_ARG;
  std::vector<HostJob> jobs(static_cast<size_t>(n));
  for (int32_t i = 0; i < n; ++i) {
    fx_status st = host_job(p, descs[i].img, descs[i].width, descs[i].height, descs[i].pitch_bytes, descs[i].dtype,
                            descs[i].out_mask, descs[i].out_pitch, &jobs[static_cast<size_t>(i)]);
    if (st != FX_OK) return st;
  }
  return host_pipeline(p, jobs.data(), n);
}

}  // extern "C"

namespace fx {
FX_CHECK_COUNTER(checked_count_plan)
}  // namespace fx
