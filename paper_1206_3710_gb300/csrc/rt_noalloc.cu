// rt_noalloc.cu -- rt_trace_noalloc: the tracer with its scratch memory in a
// fixed, file-scope device array, for callers that must not allocate.
//
// rt_trace keeps its job table, energy ledger and package counter in device
// buffers that the context grows with cudaMalloc.  Some callers cannot let a
// library call cudaMalloc: an application whose device memory is all handed
// out by its own pool or caching allocator (a cudaMalloc behind its back can
// fail, or fragment memory the pool was sized for), and code on a latency-
// critical path where the implicit device synchronisation of
// cudaMalloc/cudaFree is not acceptable.  This entry point allocates nothing:
// its scratch is the static array below, which every GPU that loads the
// library holds until the process exits.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <thread>

#include "rt_internal.cuh"

// 64 KiB: job record, 256 wavelength bins, 4 sources, ledger and counter
#define RT_NOALLOC_SCRATCH_BYTES (64 * 1024)
#define RT_NOALLOC_MAX_SOURCES 4
#define RT_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

namespace {

// Held for the whole host side of a call: the calls share the device
// scratch and the host staging area below, so they are serialised on the
// host (their kernels may still overlap on the GPU if the caller uses
// several streams; see rt.h).
std::mutex g_call_mu;
void* g_scratch_addr[RT_NOALLOC_MAX_DEVICES] = {};
// host image of the job table, uploaded at every call (a static array rather
// than a stack one: the call needs only a few hundred bytes of stack)
alignas(256) unsigned char g_host_stage[RT_NOALLOC_SCRATCH_BYTES];
long long g_pk[RT_NOALLOC_MAX_SOURCES][RT_MAX_LAMBDA];

// Poll the stream until its work is done, at most timeout seconds.  The
// upload before the launch and the read-back after it use pageable host
// memory, and such copies wait for the stream's earlier work inside the
// copy call, unbounded; polling first keeps every wait of the call bounded.
int wait_stream(cudaStream_t st, double timeout, const char* what) {
  const auto t0 = std::chrono::steady_clock::now();
  for (int spins = 0;; ++spins) {
    const cudaError_t q = cudaStreamQuery(st);
    if (q == cudaSuccess) return RT_OK;
    if (q != cudaErrorNotReady) return rtk::set_error(RT_ERR_CUDA, "rt_trace_noalloc: device error while waiting");
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout)
      return rtk::set_error(RT_ERR_TIMEOUT, what);
    if (spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// Device address of the scratch array on `device`, looked up once per device
// with that device current (in host code the array's name is only a
// host-side stand-in).
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= RT_NOALLOC_MAX_DEVICES)
    return rtk::set_error(RT_ERR_INVALID, "rt_trace_noalloc: device index out of range");
  if (!g_scratch_addr[device]) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) return rtk::set_error(RT_ERR_CUDA, "rt_trace_noalloc: cudaGetSymbolAddress failed");
    g_scratch_addr[device] = p;
  }
  *out = reinterpret_cast<unsigned char*>(g_scratch_addr[device]);
  return RT_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

extern "C" int rt_trace_noalloc(const rt_grid* grid, int n_src, const rt_source* src, const rt_optics* op,
                                const rt_trace_params* p, double* absorbed_dev, rt_ledger* ledger,
                                void* cuda_stream) {
  using namespace rtk;
  if (ledger) memset(ledger, 0, sizeof *ledger);
  if (!grid || !src || !op || !p) return set_error(RT_ERR_INVALID, "rt_trace_noalloc: NULL argument");
  if (p->split_factor > 1 || p->poly_group > 1)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: no resampling or polychromatic packages");
  if (n_src < 1 || n_src > RT_NOALLOC_MAX_SOURCES)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: n_src must be 1..4 (scratch limit)");
  if (op->n_lambda < 1 || op->n_lambda > RT_MAX_LAMBDA || !op->kappa_ext || !op->albedo || !op->g_hg)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: n_lambda must be 1..256 with non-NULL optics arrays");
  const int nl = op->n_lambda;
  for (int b = 0; b < nl; ++b)
    if (!(op->kappa_ext[b] >= 0.0) || !std::isfinite(op->kappa_ext[b]) || !(op->albedo[b] >= 0.0 && op->albedo[b] <= 1.0) ||
        !(std::fabs(op->g_hg[b]) < 1.0))
      return set_error(RT_ERR_INVALID, "rt_trace_noalloc: optics out of range");
  if (p->precision != 32 && p->precision != 64) return set_error(RT_ERR_INVALID, "rt_trace_noalloc: precision must be 32 or 64");
  if (p->estimator != RT_EST_CONTINUOUS && p->estimator != RT_EST_ANALOG)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: unknown estimator");
  if (p->packet_offset < 0) return set_error(RT_ERR_INVALID, "rt_trace_noalloc: packet_offset must be >= 0");
  if (p->rr_wmin > 0.0 && (p->estimator != RT_EST_CONTINUOUS || !(p->rr_p >= 0.0 && p->rr_p < 1.0)))
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: roulette needs the continuous estimator and rr_p in [0,1)");
  for (int s = 0; s < n_src; ++s) {
    const rt_source& S = src[s];
    if (S.kind != RT_SRC_POINT && S.kind != RT_SRC_EXTERNAL && S.kind != RT_SRC_BEAM)
      return set_error(RT_ERR_INVALID, "rt_trace_noalloc: only point, external and beam sources (a dust source needs "
                                       "a cumulative-emission table larger than the scratch)");
    if (!S.bin_energy) return set_error(RT_ERR_INVALID, "rt_trace_noalloc: bin_energy is NULL");
    for (int b = 0; b < nl; ++b)
      if (!(S.bin_energy[b] >= 0.0) || !std::isfinite(S.bin_energy[b]))
        return set_error(RT_ERR_INVALID, "rt_trace_noalloc: bin_energy must be finite and >= 0");
    if (S.kind == RT_SRC_BEAM && !(S.dir[0] * S.dir[0] + S.dir[1] * S.dir[1] + S.dir[2] * S.dir[2] > 0.0))
      return set_error(RT_ERR_INVALID, "rt_trace_noalloc: beam direction is zero");
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the call uploads from and reads back into host memory and polls the
  // stream: none of this can be captured into a graph
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess)
    return set_error(RT_ERR_CUDA, "rt_trace_noalloc: cannot query the stream");
  if (cap != cudaStreamCaptureStatusNone)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: the stream is capturing a graph");
  std::lock_guard<std::mutex> lk(g_call_mu);
  rt_grid_info gi;
  if (rt_grid_get_info(grid, &gi) != RT_OK) return RT_ERR_INVALID;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, gi.node) != cudaSuccess)
    return set_error(RT_ERR_CUDA, "rt_trace_noalloc: cannot query the grid's device");
  const int device = pa.device;

  // packages per (source, bin)
  long long (&pk)[RT_NOALLOC_MAX_SOURCES][RT_MAX_LAMBDA] = g_pk;
  double energy_tot = 0.0;
  for (int s = 0; s < n_src; ++s)
    for (int b = 0; b < nl; ++b) energy_tot += src[s].bin_energy[b];
  for (int s = 0; s < n_src; ++s)
    for (int b = 0; b < nl; ++b) {
      long long v;
      if (p->packets_per_bin > 0) v = p->packets_per_bin;
      else if (p->packets_total > 0) {
        const double e = src[s].bin_energy[b];
        v = energy_tot > 0 ? (long long)std::floor((double)p->packets_total * e / energy_tot) : 0;
        if (e > 0 && v == 0) v = 1;
      } else if (p->packets) {
        v = p->packets[s * nl + b];
        if (v < 0) return set_error(RT_ERR_INVALID, "rt_trace_noalloc: negative package count");
      } else {
        return set_error(RT_ERR_INVALID, "rt_trace_noalloc: set packets_per_bin, packets_total or packets");
      }
      pk[s][b] = v;
    }

  // scratch layout: ledger | counter | job | bins | items | prefixes | weights (f64, f32)
  const size_t o_led = 0, o_cnt = sizeof(LedgerDev);
  const size_t o_job = align_up(o_cnt + sizeof(unsigned long long), 256);
  const size_t o_bin = align_up(o_job + sizeof(JobDev), 16);
  const size_t o_item = align_up(o_bin + sizeof(BinDev) * nl, 16);
  const size_t o_pref = align_up(o_item + sizeof(ItemDev) * n_src, 16);
  const size_t o_w0 = align_up(o_pref + sizeof(long long) * (nl + 1) * n_src, 16);
  const size_t o_w0f = align_up(o_w0 + sizeof(double) * nl * n_src, 16);
  const size_t bytes = align_up(o_w0f + sizeof(float) * nl * n_src, 16);
  if (bytes > RT_NOALLOC_SCRATCH_BYTES)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: job table exceeds the 64 KiB scratch");

  unsigned char* dev = nullptr;
  int rc = scratch_address(device, &dev);
  if (rc) return rc;

  unsigned char* host = g_host_stage;
  memset(host, 0, bytes);  // ledger and package counter start at zero
  JobDev& J = *reinterpret_cast<JobDev*>(host + o_job);
  J.node = gi.node;
  J.rho64 = gi.density64;
  J.coord = gi.coord;
  J.level = gi.level;
  for (int a = 0; a < 3; ++a) J.root[a] = (uint32_t)gi.root[a];
  J.depth = gi.depth;
  J.h0 = gi.box[0] / gi.root[0];
  J.n_lambda = nl;
  J.estimator = p->estimator;
  J.bins = reinterpret_cast<const BinDev*>(dev + o_bin);
  J.n_cells = gi.n_cells;
  J.absorbed = absorbed_dev;
  J.abs_bins = p->per_lambda ? nl : 1;
  J.img_bins = J.abs_bins;
  J.packet_log = p->packet_log_dev;
  J.ledger = reinterpret_cast<LedgerDev*>(dev + o_led);
  J.seed = p->seed;
  J.job_id = p->job;
  J.iter = p->iter;
  J.rr_wmin = p->rr_wmin;
  J.rr_p = p->rr_p;
  J.step_limit = p->step_limit > 0 ? p->step_limit : 100000000ll;
  J.peel_tau_max = p->peel_tau_max;
  J.pkt_offset = p->packet_offset;
  J.rr_wmin_f = (float)p->rr_wmin;
  J.rr_p_f = (float)p->rr_p;
  J.peel_tau_max_f = (float)p->peel_tau_max;
  BinDev* B = reinterpret_cast<BinDev*>(host + o_bin);
  for (int b = 0; b < nl; ++b) {
    B[b].kext_d = op->kappa_ext[b] * J.h0;
    B[b].kext_f = (float)(op->kappa_ext[b] * J.h0 * gi.rho_scale);
    B[b].albedo = (float)op->albedo[b];
    B[b].g = (float)op->g_hg[b];
    B[b].albedo_d = op->albedo[b];
    B[b].g_d = op->g_hg[b];
  }
  ItemDev* I = reinterpret_cast<ItemDev*>(host + o_item);
  long long* pref = reinterpret_cast<long long*>(host + o_pref);
  double* w0 = reinterpret_cast<double*>(host + o_w0);
  float* w0f = reinterpret_cast<float*>(host + o_w0f);
  double w0_max = 0.0;
  long long total = 0;
  int n_items = 0;
  for (int s = 0; s < n_src; ++s) {
    long long* pr = pref + (size_t)s * (nl + 1);
    double* w = w0 + (size_t)s * nl;
    float* wf = w0f + (size_t)s * nl;
    pr[0] = 0;
    for (int b = 0; b < nl; ++b) {
      pr[b + 1] = pr[b] + pk[s][b];
      w[b] = pk[s][b] > 0 ? src[s].bin_energy[b] / (double)pk[s][b] : 0.0;
      wf[b] = (float)w[b];
      w0_max = std::max(w0_max, w[b]);
    }
    if (pr[nl] == 0) continue;
    ItemDev& it = I[n_items++];
    it.pkt_begin = total;
    it.pkt_end = total + pr[nl];
    it.log_offset = total;
    it.job = 0;
    it.kind = src[s].kind;
    it.src_index = (uint32_t)s;
    for (int a = 0; a < 3; ++a) it.pos[a] = src[s].pos[a] / J.h0;
    if (src[s].kind == RT_SRC_BEAM) {
      const double n2 = std::sqrt(src[s].dir[0] * src[s].dir[0] + src[s].dir[1] * src[s].dir[1] +
                                  src[s].dir[2] * src[s].dir[2]);
      for (int a = 0; a < 3; ++a) it.dir[a] = src[s].dir[a] / n2;
    }
    it.bin_prefix = reinterpret_cast<const long long*>(dev + o_pref) + (size_t)s * (nl + 1);
    it.W0 = reinterpret_cast<const double*>(dev + o_w0) + (size_t)s * nl;
    it.W0f = reinterpret_cast<const float*>(dev + o_w0f) + (size_t)s * nl;
    for (int a = 0; a < 3; ++a) {
      it.posf[a] = (float)it.pos[a];
      it.dirf[a] = (float)it.dir[a];
    }
    it.dust_first = nullptr;
    total += pr[nl];
  }
  J.led_shift = ledger_shift(w0_max, p->rr_wmin, p->rr_p);
  if (p->packet_log_dev && total > p->packet_log_rows)
    return set_error(RT_ERR_INVALID, "rt_trace_noalloc: packet_log_rows is smaller than the launch's packages");

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  auto restore = [&](int code) {
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return code;
  };
  const double timeout = p->timeout_s > 0 ? p->timeout_s : 3600.0;
  rc = wait_stream(st, timeout, "rt_trace_noalloc: earlier work on the stream did not finish in time");
  if (rc) return restore(rc);
  if (cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return restore(set_error(RT_ERR_CUDA, "rt_trace_noalloc: upload of the job table failed"));
  if (total > 0) {
    int sms = 0, occ = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int block = p->block_size > 0 ? p->block_size : 256;
    if (block % 32 || block > 256) return restore(set_error(RT_ERR_INVALID, "rt_trace_noalloc: bad block_size"));
    if (trace_occupancy(p->precision, false, block, &occ) != cudaSuccess || occ < 1) occ = 1;
    if (p->blocks_per_sm > 0 && p->blocks_per_sm < occ) occ = p->blocks_per_sm;
    LaunchCfg cfg;
    cfg.block = block;
    cfg.blocks = sms * occ;
    cfg.blocks_tiled = cfg.blocks;  // untiled only
    cfg.refill = p->refill_threshold > 0 ? (p->refill_threshold > 32 ? 32 : p->refill_threshold) : 8;
    PeelQueue q;  // no observers: no peel-off queue
    q.rec = nullptr;
    q.count = nullptr;
    q.cap = 0;
    if (launch_trace(p->precision, false, p->estimator, false, reinterpret_cast<const JobDev*>(dev + o_job),
                     reinterpret_cast<const ItemDev*>(dev + o_item), n_items,
                     reinterpret_cast<unsigned long long*>(dev + o_cnt), total, cfg, q, st) != cudaSuccess)
      return restore(set_error(RT_ERR_CUDA, "rt_trace_noalloc: kernel launch failed"));
  }
  // bounded wait on the stream (no event objects), then the ledger: the
  // copy is issued only once the kernel has finished, so a timeout leaves
  // no copy pending into this call's memory
  rc = wait_stream(st, timeout, "rt_trace_noalloc: device work did not finish in time");
  if (rc) return restore(rc);
  LedgerDev hl;
  if (cudaMemcpyAsync(&hl, dev + o_led, sizeof hl, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return restore(set_error(RT_ERR_CUDA, "rt_trace_noalloc: ledger read-back failed"));
  if (ledger) {
    ledger->emitted = hl.emitted;
    ledger->absorbed = hl.absorbed;
    ledger->escaped = hl.escaped;
    ledger->rr_gain = hl.rr_gain;
    ledger->rr_loss = hl.rr_loss;
    ledger->killed = hl.killed;
    ledger->peeled = hl.peeled;
    ledger->n_packets = hl.n_packets;
    ledger->n_cross = hl.n_cross;
    ledger->n_scatter = hl.n_scatter;
    ledger->n_peel_cross = hl.n_peel_cross;
    ledger->n_killed = hl.n_killed;
    ledger->n_peel_out = hl.n_peel_out;
    ledger->n_peel_deferred = hl.n_peel_deferred;
    ledger->status = hl.status ? RT_ERR_STEP_LIMIT : RT_OK;
    ledger->kernel_ms = 0.0;
    ledger->n_launches = total > 0 ? 1 : 0;
  }
  if (hl.status) return restore(set_error(RT_ERR_STEP_LIMIT, "rt_trace_noalloc: some packages hit the step limit"));
  return restore(RT_OK);
}
