// Continuous-batching render server.
//
// One host thread owns a CUDA stream and a device pool of rays.  Every
// iteration it (1) admits pending requests while a request slot, a
// contiguous pixel range of the pool and the device-memory budget are free,
// generating their rays straight into the shared active-ray list; (2) runs
// one march step (decoder queries + converge/step/compact) over the active
// rays of all in-flight requests together; (3) counts each request's
// remaining active rays and finishes every request whose rays are all done:
// L1 depth loss and latent gradient for render+backward requests, then the
// copy of its results to the caller's host buffers.  A request joins the
// batch at the next step after a slot frees up and leaves as soon as its own
// rays are done, so requests of different sizes overlap on the device.
// Each ray's arithmetic does not depend on which other rays share its step,
// so a request's result is the same alone and in the mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "step.cuh"

namespace dist {
namespace {

enum ReqState { kPending, kRunning, kDone, kFailed };

struct Req {
  uint64_t ticket = 0;
  dist_request r;
  std::vector<float> z;
  int slot = -1;
  long long off = 0, n = 0;
  size_t bytes = 0;
  ReqState state = kPending;
  dist_status err = DIST_OK;
};

// Requests per slot among the listed rays (camera index == slot), with a
// shared-memory histogram per block.
__global__ void count_slots_kernel(const int* l0, const int* c0, const int* l1, const int* c1,
                                   const int* l2, const int* c2, const float4* st, int n_slots,
                                   int* active) {
  extern __shared__ int hist[];
  for (int s = threadIdx.x; s < n_slots; s += blockDim.x) hist[s] = 0;
  __syncthreads();
  const int n0 = *c0, n1 = *c1, n2 = *c2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n0 + n1 + n2;
       j += gridDim.x * blockDim.x) {
    const int ray = j < n0 ? l0[j] : (j < n0 + n1 ? l1[j - n0] : l2[j - n0 - n1]);
    atomicAdd(&hist[__float_as_int(st[ray].w)], 1);
  }
  __syncthreads();
  for (int s = threadIdx.x; s < n_slots; s += blockDim.x)
    if (hist[s]) atomicAdd(&active[s], hist[s]);
}

size_t bytes_per_pixel(int K) {
  // ray state (incl. the refinement samples), lists, MLP outputs, per-pixel
  // outputs, target, upstream gradient and backward probes
  return 16 + 16 + 12 + 24 + 12 + (4 + 4 + 1 + 4 + 4 + 4 + 8 * K) + 4 + 4 + (16 + 16 + 4);
}

}  // namespace
}  // namespace dist

using namespace dist;

struct dist_server {
  const dist_decoder* dec = nullptr;
  dist_trace_params p;
  long long max_rays = 0;
  size_t budget = 0;
  int max_req = 0;
  int L = 0;
  cudaStream_t st = nullptr;
  // device pool
  float4* dir = nullptr;
  float4* stt = nullptr;
  int* fq = nullptr;
  float* fprev = nullptr;
  float* dprev = nullptr;
  int* act[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  float* fbuf[3] = {nullptr, nullptr, nullptr};
  int* cnt = nullptr;             // [parity][list 0, 1], then [parity] of list 2 (FP16 stage)
  CamDev* cams = nullptr;         // [max_req]
  float* z = nullptr;             // [max_req][L]
  float* bfold = nullptr;         // [2][max_req][512]
  double* gacc = nullptr;         // [2][max_req][512]
  float *depth = nullptr, *sil = nullptr, *d_hit = nullptr, *d_min = nullptr, *f_min = nullptr;
  float *tgt = nullptr, *g_depth = nullptr, *dz = nullptr;
  uint8_t* mask = nullptr;
  int32_t *steps = nullptr, *status = nullptr;
  float4 *pp = nullptr, *pq = nullptr;
  int *pix = nullptr, *pcount = nullptr, *icnt = nullptr, *slot_active = nullptr;
  int* slot_active_host = nullptr;
  double* loss = nullptr;
  unsigned long long* queries = nullptr;
  void* tc_scratch = nullptr;
  void* wide_scratch = nullptr;
  unsigned long long step_seq = 0;   // sequence number of the last fused step
  std::vector<void*> allocs;
  // host state
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;
  std::vector<int> free_slots;
  std::map<long long, long long> free_ranges;   // offset -> length
  std::vector<Req*> running;                    // by slot
  size_t used_bytes = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  bool exited = false;
  dist_status dead = DIST_OK;
  int par = 0;
  std::thread th;

  RayPool pool() const {
    RayPool P;
    P.cams = cams; P.st = stt; P.dir = dir; P.fq = fq; P.fprev = fprev; P.dprev = dprev;
    P.refine = is_tc(p.precision) ? p.refine_steps : 0;
    P.secant = is_tc(p.precision) && p.refine_rule == DIST_REFINE_SECANT ? 1 : 0;
    P.alpha_fp32 = (is_tc(p.precision) && p.alpha_refine > 0.f) ? p.alpha_refine : p.alpha;
    std::memset(&P.o, 0, sizeof(P.o));
    P.o.depth = depth; P.o.sil = sil; P.o.mask = mask; P.o.steps = steps; P.o.status = status;
    P.o.d_hit = d_hit; P.o.d_min = d_min; P.o.f_min = f_min; P.o.queries = queries;
    P.K = p.k_min; P.eps = p.eps; P.alpha = p.alpha; P.eps_bf16 = p.eps_bf16;
    P.eps_mid = p.precision == DIST_PREC_BF16 ? p.eps_mid : 0.f;
    P.radius = p.radius; P.max_steps = p.max_steps;
    return P;
  }

  bool take_range(long long n, long long* off) {
    for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const long long rest = it->second - n;
        const long long start = it->first + n;
        free_ranges.erase(it);
        if (rest > 0) free_ranges[start] = rest;
        return true;
      }
    }
    return false;
  }

  void give_range(long long off, long long n) {
    auto it = free_ranges.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_ranges.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_ranges.erase(nx);
    }
    if (it != free_ranges.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_ranges.erase(it);
      }
    }
  }

  dist_status admit(bool* any) {
    std::vector<Req*> now;
    {
      std::lock_guard<std::mutex> lock(mu);
      while (!pending.empty()) {
        Req* R = pending.front();
        long long off = 0;
        if (free_slots.empty() || used_bytes + R->bytes > budget) break;
        if (!take_range(R->n, &off)) break;
        pending.pop_front();
        R->slot = free_slots.back();
        free_slots.pop_back();
        R->off = off;
        R->state = kRunning;
        used_bytes += R->bytes;
        running[R->slot] = R;
        now.push_back(R);
      }
    }
    *any = !now.empty();
    const int first = is_tc(p.precision) ? 0 : 1;
    const RayPool P = pool();
    for (Req* R : now) {
      CamDev c;
      std::memset(&c, 0, sizeof(c));
      std::memcpy(c.c, R->r.cam.c, sizeof(c.c));
      std::memcpy(c.R, R->r.cam.R, sizeof(c.R));
      c.fx = R->r.cam.fx; c.fy = R->r.cam.fy; c.cx = R->r.cam.cx; c.cy = R->r.cam.cy;
      c.H = R->r.cam.H; c.W = R->r.cam.W; c.shape = R->slot; c.offset = R->off;
      DIST_CUDA_TRY(pool_write_cam(c, R->slot, cams, st));
      DIST_CUDA_TRY(cudaMemcpyAsync(z + (size_t)R->slot * L, R->z.data(), L * sizeof(float),
                                    cudaMemcpyHostToDevice, st));
      if (R->r.kind == DIST_REQ_RENDER_BACKWARD)
        DIST_CUDA_TRY(cudaMemcpyAsync(tgt + R->off, R->r.tgt_depth, R->n * sizeof(float),
                                      cudaMemcpyHostToDevice, st));
      DIST_CUDA_TRY(pool_raygen(P, R->slot, R->off, R->n, act[par][first], cnt + 2 * par + first,
                                st));
    }
    if (!now.empty())
      DIST_CUDA_TRY(launch_fold_bias(dec->f32, z, max_req, bfold, bfold + (size_t)max_req * 512, st));
    return DIST_OK;
  }

  dist_status step() {
    const RayPool P = pool();
    const float* b0 = bfold;
    const float* bs = bfold + (size_t)max_req * 512;
    RowSrc src{};
    src.st = stt; src.dir = dir; src.cams = cams;
    RowSrc sx = src;
    sx.count = cnt + 2 * par + 1;
    sx.idx = act[par][1];
    RowSrc sm = src;                 // FP16 stage of a BF16 march (list 2)
    sm.count = cnt + 4 + par;
    sm.idx = act[par][2];
    int* out[2] = {act[par ^ 1][0], act[par ^ 1][1]};
    DIST_CUDA_TRY(cudaMemsetAsync(cnt + 2 * (par ^ 1), 0, 2 * sizeof(int), st));
    DIST_CUDA_TRY(cudaMemsetAsync(cnt + 4 + (par ^ 1), 0, sizeof(int), st));
    if (fp32_on_tc(p)) {
      // every list in one launch (an empty 16-bit list for FP32_TC), which
      // also applies the step update
      src.count = cnt + 2 * par;
      src.idx = act[par][0];
      StepFuse sf;
      pool_step_fuse(P, cnt + 2 * (par ^ 1), out, &sf);
      sf.out[2] = act[par ^ 1][2];
      sf.cnt_out[2] = cnt + 4 + (par ^ 1);
      if (p.latency_mode) {
        sf.wide = static_cast<uint8_t*>(wide_scratch);
        sf.seq_flag = tc_wide_seq_flag(wide_scratch);
        sf.seq = ++step_seq;
      }
      DIST_CUDA_TRY(mlp_tc_fused(dec, src, fbuf[0], sx, fbuf[1], b0, bs, st,
                                 p.precision == DIST_PREC_FP16, &sf,
                                 P.eps_mid > 0.f ? &sm : nullptr, fbuf[2]));
    } else {
      if (is_tc(p.precision)) {
        src.count = cnt + 2 * par;
        src.idx = act[par][0];
        DIST_CUDA_TRY(mlp_tc_forward(dec, src, b0, bs, fbuf[0], st,
                                     p.precision == DIST_PREC_FP16));
      }
      DIST_CUDA_TRY(mlp_fp32_forward(dec->f32, sx, b0, bs, fbuf[1], st, is_tc(p.precision)));
      int* in[2] = {act[par][0], act[par][1]};
      const float* f[2] = {fbuf[0], fbuf[1]};
      DIST_CUDA_TRY(pool_step(P, cnt + 2 * par, cnt + 2 * (par ^ 1), in, f, out, st));
    }
    par ^= 1;
    DIST_CUDA_TRY(cudaMemsetAsync(slot_active, 0, max_req * sizeof(int), st));
    count_slots_kernel<<<num_sms(), 256, max_req * sizeof(int), st>>>(
        act[par][0], cnt + 2 * par, act[par][1], cnt + 2 * par + 1, act[par][2], cnt + 4 + par,
        stt, max_req, slot_active);
    count_launch(1);
    DIST_CUDA_TRY(cudaGetLastError());
    DIST_CUDA_TRY(cudaMemcpyAsync(slot_active_host, slot_active, max_req * sizeof(int),
                                  cudaMemcpyDeviceToHost, st));
    DIST_CUDA_TRY(cudaStreamSynchronize(st));
    for (int s = 0; s < max_req; ++s) {
      Req* R = running[s];
      if (R && slot_active_host[s] == 0) {
        dist_status e = finish(R);
        if (e != DIST_OK) return e;
      }
    }
    return DIST_OK;
  }

  dist_status finish(Req* R) {
    const RayPool P = pool();
    const int s = R->slot;
    if (R->r.kind == DIST_REQ_RENDER_BACKWARD) {
      // accumulator tables are [slot][width], as the adjoint kernel indexes them
      const size_t w = (size_t)dec->f32.width;
      double* G0 = gacc;
      double* Gs = gacc + (size_t)max_req * 512;
      DIST_CUDA_TRY(pool_loss_depth(R->n, depth + R->off, mask + R->off, tgt + R->off, loss + s,
                                    g_depth + R->off, icnt, st));
      DIST_CUDA_TRY(cudaMemsetAsync(G0 + s * w, 0, w * sizeof(double), st));
      DIST_CUDA_TRY(cudaMemsetAsync(Gs + s * w, 0, w * sizeof(double), st));
      DIST_CUDA_TRY(cudaMemsetAsync(pcount, 0, sizeof(int), st));
      DIST_CUDA_TRY(pool_probes_depth(P, s, R->off, R->n, g_depth, pp, pq, pix, pcount, st));
      // the adjoint in the march's precision, as dist_trace_bwd does
      if (is_tc(p.precision))
        DIST_CUDA_TRY(mlp_tc_adjoint(dec, pp, pq, pcount, bfold, bfold + (size_t)max_req * 512,
                                     nullptr, G0, Gs, 1, tc_scratch, st,
                                     p.precision == DIST_PREC_FP16));
      else if (p.precision == DIST_PREC_FP32_TC)
        DIST_CUDA_TRY(mlp_tcx_adjoint(dec, pp, pq, pcount, bfold, bfold + (size_t)max_req * 512,
                                      nullptr, G0, Gs, 1, tc_scratch, st));
      else
        DIST_CUDA_TRY(mlp_fp32_adjoint(dec->f32, pp, pq, pcount, bfold,
                                       bfold + (size_t)max_req * 512, nullptr, G0, Gs, 1, st));
      DIST_CUDA_TRY(cudaMemsetAsync(dz + (size_t)s * L, 0, L * sizeof(float), st));
      DIST_CUDA_TRY(pool_latent_finalize(dec->f32, G0 + s * w, Gs + s * w, dz + (size_t)s * L, st));
      DIST_CUDA_TRY(cudaMemcpyAsync(R->r.dz, dz + (size_t)s * L, L * sizeof(float),
                                    cudaMemcpyDeviceToHost, st));
      DIST_CUDA_TRY(cudaMemcpyAsync(R->r.loss, loss + s, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    DIST_CUDA_TRY(cudaMemcpyAsync(R->r.depth, depth + R->off, R->n * sizeof(float),
                                  cudaMemcpyDeviceToHost, st));
    if (R->r.sil)
      DIST_CUDA_TRY(cudaMemcpyAsync(R->r.sil, sil + R->off, R->n * sizeof(float),
                                    cudaMemcpyDeviceToHost, st));
    if (R->r.mask)
      DIST_CUDA_TRY(cudaMemcpyAsync(R->r.mask, mask + R->off, R->n, cudaMemcpyDeviceToHost, st));
    DIST_CUDA_TRY(cudaStreamSynchronize(st));
    std::lock_guard<std::mutex> lock(mu);
    running[s] = nullptr;
    free_slots.push_back(s);
    give_range(R->off, R->n);
    used_bytes -= R->bytes;
    R->state = kDone;
    return DIST_OK;
  }

  void fail_all(dist_status e) {
    std::lock_guard<std::mutex> lock(mu);
    dead = e;
    for (Req* R : pending) { R->state = kFailed; R->err = e; }
    pending.clear();
    for (Req*& R : running)
      if (R) { R->state = kFailed; R->err = e; R = nullptr; }
  }

  void loop() {
    cudaSetDevice(device);
    for (;;) {
      bool have_work = false;
      {
        std::unique_lock<std::mutex> lock(mu);
        if (stop) break;
        bool run = false;
        for (Req* R : running) run |= R != nullptr;
        if (!run && pending.empty()) {
          cv.wait_for(lock, std::chrono::milliseconds(2));
          continue;
        }
        have_work = run || !pending.empty();
      }
      if (!have_work) continue;
      DIST_NVTX("serve iteration");
      bool any = false;
      dist_status e = admit(&any);
      bool run = false;
      {
        std::lock_guard<std::mutex> lock(mu);
        for (Req* R : running) run |= R != nullptr;
      }
      if (e == DIST_OK && run) e = step();
      if (e != DIST_OK) {
        fail_all(e);
        break;
      }
      if (!run && !any) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    std::lock_guard<std::mutex> lock(mu);
    exited = true;
    cv.notify_all();
  }

  int device = 0;
};

namespace {

dist_status server_alloc(dist_server* S, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    set_error(std::string("dist_serve_create: cudaMalloc: ") + cudaGetErrorString(e));
    return DIST_E_NOMEM;
  }
  S->allocs.push_back(*p);
  return DIST_OK;
}

void server_free(dist_server* S) {
  for (void* p : S->allocs) cudaFree(p);
  if (S->slot_active_host) cudaFreeHost(S->slot_active_host);
  if (S->st) cudaStreamDestroy(S->st);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}

}  // namespace

extern "C" {

dist_status dist_serve_create(const dist_decoder* dec, const dist_trace_params* p,
                              int64_t max_rays, size_t mem_budget, int max_requests,
                              dist_server** out) {
  DIST_CHECK(dec && p && out, DIST_E_INVALID, "dist_serve_create: NULL argument");
  DIST_CHECK(is_sdf_decoder(dec->desc), DIST_E_INVALID,
             "dist_serve_create needs an SDF decoder (out_dim 1, latent_dim0 = latent_dim)");
  DIST_CHECK(max_rays >= 1 && max_rays <= (1ll << 28), DIST_E_INVALID,
             "dist_serve_create: max_rays out of range");
  DIST_CHECK(max_requests >= 1 && max_requests <= kMaxShapes, DIST_E_INVALID,
             "dist_serve_create: max_requests must be 1..1024");
  DIST_CHECK(p->max_steps >= 1 && p->k_min >= 1 && p->k_min <= kMaxK && p->eps > 0.f &&
                 p->alpha > 0.f && p->radius > 0.f,
             DIST_E_INVALID, "dist_serve_create: bad trace parameters");
  DIST_CHECK(valid_precision(p->precision), DIST_E_INVALID, "dist_serve_create: bad precision");
  DIST_CHECK(p->refine_engine == DIST_REFINE_TC || p->refine_engine == DIST_REFINE_SIMT,
             DIST_E_INVALID, "dist_serve_create: bad refine_engine");
  DIST_CHECK(p->refine_rule == DIST_REFINE_MARCH || p->refine_rule == DIST_REFINE_SECANT,
             DIST_E_INVALID, "dist_serve_create: bad refine_rule");
  DIST_CHECK(!(is_tc(p->precision) || fp32_on_tc(*p)) || dec->tc.ok, DIST_E_UNSUPPORTED,
             "the tensor-core decoder covers only the DeepSDF shape");
  DIST_CHECK(p->coarse_levels == 0, DIST_E_INVALID,
             "dist_serve_create: coarse-to-fine tracing is not supported by the server");
  DIST_CHECK(p->precision != DIST_PREC_BF16 || p->eps_mid == 0.f ||
                 (p->eps_mid > 0.f && p->eps_mid < p->eps_bf16 && fp32_on_tc(*p) &&
                  p->refine_steps == 0 && p->refine_rule == DIST_REFINE_MARCH),
             DIST_E_INVALID,
             "dist_serve_create: eps_mid must be 0, or in (0, eps_bf16) with the TC refine "
             "engine, refine_steps 0 and the MARCH rule");
  dist_server* S = new dist_server();
  S->dec = dec;
  S->p = *p;
  S->max_rays = max_rays;
  S->budget = mem_budget;
  S->max_req = max_requests;
  S->L = dec->f32.latent;
  cudaGetDevice(&S->device);
  const size_t n = (size_t)max_rays;
  const int K = p->k_min;
  dist_status s = DIST_OK;
  void* q = nullptr;
#define SV_ALLOC(field, bytes)                                   \
  if (s == DIST_OK) {                                            \
    s = server_alloc(S, &q, (bytes));                            \
    S->field = reinterpret_cast<decltype(S->field)>(q);          \
  }
  SV_ALLOC(dir, n * sizeof(float4));
  SV_ALLOC(stt, n * sizeof(float4));
  SV_ALLOC(fq, n * sizeof(int));
  SV_ALLOC(fprev, n * sizeof(float));
  SV_ALLOC(dprev, n * sizeof(float));
  SV_ALLOC(act[0][0], n * sizeof(int));
  SV_ALLOC(act[0][1], n * sizeof(int));
  SV_ALLOC(act[1][0], n * sizeof(int));
  SV_ALLOC(act[1][1], n * sizeof(int));
  SV_ALLOC(act[0][2], n * sizeof(int));
  SV_ALLOC(act[1][2], n * sizeof(int));
  SV_ALLOC(fbuf[0], n * sizeof(float));
  SV_ALLOC(fbuf[1], n * sizeof(float));
  SV_ALLOC(fbuf[2], n * sizeof(float));
  SV_ALLOC(cnt, 6 * sizeof(int));
  SV_ALLOC(cams, (size_t)max_requests * sizeof(CamDev));
  SV_ALLOC(z, (size_t)max_requests * S->L * sizeof(float));
  SV_ALLOC(bfold, (size_t)2 * max_requests * 512 * sizeof(float));
  SV_ALLOC(gacc, (size_t)2 * max_requests * 512 * sizeof(double));
  SV_ALLOC(depth, n * sizeof(float));
  SV_ALLOC(sil, n * sizeof(float));
  SV_ALLOC(d_hit, n * sizeof(float));
  SV_ALLOC(d_min, n * K * sizeof(float));
  SV_ALLOC(f_min, n * K * sizeof(float));
  SV_ALLOC(tgt, n * sizeof(float));
  SV_ALLOC(g_depth, n * sizeof(float));
  SV_ALLOC(dz, (size_t)max_requests * S->L * sizeof(float));
  SV_ALLOC(mask, n);
  SV_ALLOC(steps, n * sizeof(int32_t));
  SV_ALLOC(status, n * sizeof(int32_t));
  SV_ALLOC(pp, n * sizeof(float4));
  SV_ALLOC(pq, n * sizeof(float4));
  SV_ALLOC(pix, n * sizeof(int));
  SV_ALLOC(pcount, sizeof(int));
  SV_ALLOC(icnt, sizeof(int));
  SV_ALLOC(slot_active, max_requests * sizeof(int));
  SV_ALLOC(loss, max_requests * sizeof(double));
  SV_ALLOC(queries, 2 * sizeof(unsigned long long));
  SV_ALLOC(tc_scratch, (size_t)num_sms() * kTcAdjScratchPerCta);
  SV_ALLOC(wide_scratch, tc_wide_scratch_bytes());
#undef SV_ALLOC
  if (s == DIST_OK &&
      cudaMemset(tc_wide_seq_flag(S->wide_scratch), 0, sizeof(unsigned long long)) != cudaSuccess) {
    set_error("dist_serve_create: cudaMemset failed");
    s = DIST_E_CUDA;
  }
  if (s == DIST_OK && cudaMallocHost(&S->slot_active_host, max_requests * sizeof(int)) != cudaSuccess) {
    S->slot_active_host = nullptr;
    set_error("dist_serve_create: cudaMallocHost failed");
    s = DIST_E_NOMEM;
  }
  if (s == DIST_OK && cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
    S->st = nullptr;
    set_error("dist_serve_create: cudaStreamCreate failed");
    s = DIST_E_CUDA;
  }
  if (s == DIST_OK) {
    cudaError_t e = cudaMemset(S->cnt, 0, 6 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(S->queries, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(S->z, 0, (size_t)max_requests * S->L * sizeof(float));
    if (e != cudaSuccess) {
      set_error(std::string("dist_serve_create: ") + cudaGetErrorString(e));
      s = DIST_E_CUDA;
    }
  }
  if (s != DIST_OK) {
    server_free(S);
    return s;
  }
  S->running.assign(max_requests, nullptr);
  for (int i = max_requests - 1; i >= 0; --i) S->free_slots.push_back(i);
  S->free_ranges[0] = max_rays;
  S->th = std::thread([S] { S->loop(); });
  *out = S;
  return DIST_OK;
}

dist_status dist_serve_submit(dist_server* S, const dist_request* r, uint64_t* ticket) {
  DIST_CHECK(S && r && ticket, DIST_E_INVALID, "dist_serve_submit: NULL argument");
  DIST_CHECK(r->kind == DIST_REQ_RENDER || r->kind == DIST_REQ_RENDER_BACKWARD, DIST_E_INVALID,
             "dist_serve_submit: bad request kind");
  DIST_CHECK(r->z && r->depth, DIST_E_INVALID, "dist_serve_submit: z and depth are required");
  DIST_CHECK(r->kind == DIST_REQ_RENDER || (r->tgt_depth && r->dz && r->loss), DIST_E_INVALID,
             "dist_serve_submit: render+backward needs tgt_depth, dz and loss");
  const dist_camera& c = r->cam;
  DIST_CHECK(c.H > 0 && c.W > 0 && c.fx != 0.f && c.fy != 0.f, DIST_E_INVALID,
             "dist_serve_submit: bad camera");
  const double cc = (double)c.c[0] * c.c[0] + (double)c.c[1] * c.c[1] + (double)c.c[2] * c.c[2];
  DIST_CHECK(cc > (double)S->p.radius * S->p.radius, DIST_E_INVALID,
             "dist_serve_submit: camera inside the bounding sphere");
  const long long n = (long long)c.H * c.W;
  const size_t bytes = (size_t)n * bytes_per_pixel(S->p.k_min);
  DIST_CHECK(n <= S->max_rays && bytes <= S->budget, DIST_E_NOMEM,
             "dist_serve_submit: request larger than the ray pool or the memory budget");
  Req* R = new Req();
  R->r = *r;
  R->z.assign(r->z, r->z + S->L);
  R->n = n;
  R->bytes = bytes;
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->dead != DIST_OK) {
    delete R;
    set_error("dist_serve_submit: server stopped after a device error");
    return S->dead;
  }
  if ((int)S->pending.size() >= 4 * S->max_req) {
    delete R;
    set_error("dist_serve_submit: pending queue full");
    return DIST_E_BUSY;
  }
  R->ticket = S->next_ticket++;
  S->pending.push_back(R);
  S->reqs[R->ticket] = R;
  *ticket = R->ticket;
  S->cv.notify_all();
  return DIST_OK;
}

dist_status dist_serve_poll(dist_server* S, uint64_t ticket, int* done) {
  DIST_CHECK(S && done, DIST_E_INVALID, "dist_serve_poll: NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  DIST_CHECK(it != S->reqs.end(), DIST_E_INVALID, "dist_serve_poll: unknown ticket");
  Req* R = it->second;
  *done = 0;
  if (R->state == kDone || R->state == kFailed) {
    const dist_status e = R->state == kDone ? DIST_OK : R->err;
    *done = 1;
    S->reqs.erase(it);
    delete R;
    if (e != DIST_OK) set_error("dist_serve_poll: request failed on the device");
    return e;
  }
  return DIST_OK;
}

dist_status dist_serve_destroy(dist_server* S) {
  if (!S) return DIST_OK;
  {
    std::unique_lock<std::mutex> lock(S->mu);
    S->stop = true;
    S->cv.notify_all();
    S->cv.wait_for(lock, std::chrono::seconds(30), [S] { return S->exited; });
    if (!S->exited) {
      // the loop is stuck in a device call: leave it and its memory behind
      S->th.detach();
      set_error("dist_serve_destroy: server thread did not stop within 30 s");
      return DIST_E_TIMEOUT;
    }
  }
  S->th.join();
  cudaStreamSynchronize(S->st);
  server_free(S);
  return DIST_OK;
}

}  // extern "C"
