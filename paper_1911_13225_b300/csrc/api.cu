// Library bookkeeping: errors, defaults, decoder upload/repacking, workspaces.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace dist {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// SM count of the device current at the first call (the library drives one
// device per process); the static's initialisation is thread-safe.
int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 148;
  }();
  return n;
}

static dist_status dev_alloc(std::vector<void*>& list, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return DIST_E_NOMEM;
  }
  list.push_back(*p);
  return DIST_OK;
}

template <class T>
static dist_status upload(std::vector<void*>& list, const T** dst, const std::vector<T>& host) {
  void* p = nullptr;
  dist_status s = dev_alloc(list, &p, host.size() * sizeof(T));
  if (s != DIST_OK) return s;
  cudaError_t e = cudaMemcpy(p, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    return DIST_E_CUDA;
  }
  *dst = static_cast<const T*>(p);
  return DIST_OK;
}

dist_status pack_tc(dist_decoder* d, const float* const* W, const float* const* b);   // mlp_tc.cu

}  // namespace dist

using namespace dist;

extern "C" {

const char* dist_last_error(void) { return g_last_error.c_str(); }

const char* dist_version(void) { return "libdist 0.1 (sm_103a)"; }

void dist_trace_params_default(dist_trace_params* p) {
  if (!p) return;
  p->max_steps = 50;
  p->eps = 5e-5f;
  p->alpha = 1.5f;
  p->k_min = 1;
  p->normal_delta = 0.f;
  p->grad_mode = DIST_GRAD_EXACT;
  p->precision = DIST_PREC_FP32;
  p->eps_bf16 = 1e-3f;
  p->radius = 1.f;
  p->refine_steps = 0;
  p->alpha_refine = 0.f;
  p->refine_engine = DIST_REFINE_TC;
  p->refine_rule = DIST_REFINE_MARCH;
  p->coarse_levels = 0;
  p->coarse_every = 3;
  p->latency_mode = 1;
  p->eps_mid = 0.f;
}

dist_status dist_decoder_create(const dist_decoder_desc* desc, const float* const* W,
                                const float* const* b, dist_decoder** out) {
  DIST_CHECK(desc && W && b && out, DIST_E_INVALID, "dist_decoder_create: NULL argument");
  const int L = desc->latent_dim, Wd = desc->width, H = desc->n_hidden, S = desc->skip;
  const int L0 = desc->latent_dim0 ? desc->latent_dim0 : L;
  const int OD = desc->out_dim ? desc->out_dim : 1;
  DIST_CHECK(OD == 1 || OD == 3, DIST_E_INVALID, "dist_decoder_create: out_dim must be 1 or 3");
  DIST_CHECK(L0 >= L && L0 <= 1024, DIST_E_INVALID,
             "dist_decoder_create: latent_dim0 must be latent_dim..1024");
  DIST_CHECK(Wd == 128 || Wd == 256 || Wd == 384 || Wd == 512, DIST_E_INVALID,
             "dist_decoder_create: width must be 128, 256, 384 or 512");
  DIST_CHECK(H >= 2 && H <= 16, DIST_E_INVALID, "dist_decoder_create: n_hidden must be 2..16");
  DIST_CHECK(L >= 1 && L + 3 <= Wd, DIST_E_INVALID, "dist_decoder_create: bad latent_dim");
  DIST_CHECK(S == -1 || (S >= 1 && S < H), DIST_E_INVALID, "dist_decoder_create: bad skip");
  DIST_CHECK(S == -1 || Wd - L - 3 >= 4, DIST_E_INVALID,
             "dist_decoder_create: skip needs width - latent_dim - 3 >= 4");
  for (int l = 0; l <= H; ++l)
    DIST_CHECK(W[l] && b[l], DIST_E_INVALID, "dist_decoder_create: NULL layer pointer");

  dist_decoder* d = new dist_decoder();
  d->desc = *desc;
  DecoderF32& f = d->f32;
  std::memset(&f, 0, sizeof(f));
  f.width = Wd; f.n_hidden = H; f.skip = S; f.latent = L;
  f.latent0 = L0; f.out_dim = OD;
  auto in_dim = [&](int l) { return (l == 0) ? L0 + 3 : Wd; };
  auto out_dim = [&](int l) { return (S > 0 && l == S - 1) ? Wd - L - 3 : Wd; };
  dist_status st = DIST_OK;
  std::vector<float> Wx0(Wd * 4, 0.f), Wxs(Wd * 4, 0.f), Wz0((size_t)Wd * L0, 0.f),
      Wzs((size_t)Wd * L, 0.f);
  for (int l = 0; l < H && st == DIST_OK; ++l) {
    const int K = in_dim(l), N = out_dim(l);
    // h-part column range of W_l: layer 0 has none; the skip layer's h part
    // is its first width - L - 3 columns; other layers read all of h.
    int kh = (l == 0) ? 0 : (l == S ? Wd - L - 3 : K);
    f.kh[l] = kh;
    f.nout[l] = N;
    std::vector<float> Wt((size_t)Wd * Wd, 0.f), Wb((size_t)Wd * Wd, 0.f), bb(Wd, 0.f);
    for (int j = 0; j < N; ++j) {
      for (int k = 0; k < kh; ++k) {
        const float w = W[l][(size_t)j * K + k];
        Wt[(size_t)k * Wd + j] = w;
        Wb[(size_t)j * Wd + k] = w;
      }
      bb[j] = b[l][j];
      if (l == 0 || l == S) {
        const int zc = kh;          // latent columns start after the h part
        std::vector<float>& Wx = (l == 0) ? Wx0 : Wxs;
        std::vector<float>& Wz = (l == 0) ? Wz0 : Wzs;
        const int Lz = (l == 0) ? L0 : L;   // code columns of this layer
        for (int k = 0; k < Lz; ++k) Wz[(size_t)j * Lz + k] = W[l][(size_t)j * K + zc + k];
        for (int a = 0; a < 3; ++a) Wx[j * 4 + a] = W[l][(size_t)j * K + zc + Lz + a];
      }
    }
    if (st == DIST_OK) st = upload(d->allocations, &f.Wt[l], Wt);
    if (st == DIST_OK) st = upload(d->allocations, &f.Wb[l], Wb);
    if (st == DIST_OK) st = upload(d->allocations, &f.b[l], bb);
  }
  if (st == DIST_OK) st = upload(d->allocations, &f.Wx0, Wx0);
  if (st == DIST_OK) st = upload(d->allocations, &f.Wxs, Wxs);
  if (st == DIST_OK) st = upload(d->allocations, &f.Wz0, Wz0);
  if (st == DIST_OK) st = upload(d->allocations, &f.Wzs, Wzs);
  if (st == DIST_OK) {
    std::vector<float> wh((size_t)OD * Wd, 0.f);
    for (int o = 0; o < OD; ++o)
      for (int k = 0; k < Wd; ++k) wh[(size_t)o * Wd + k] = W[H][(size_t)o * Wd + k];
    st = upload(d->allocations, &f.w_head, wh);
    f.b_head = b[H][0];
    for (int o = 0; o < OD; ++o) f.b_out[o] = b[H][o];
  }
  d->tc.ok = false;
  if (st == DIST_OK && Wd == 512 && H == 8 && S == 4 && L == 256) st = pack_tc(d, W, b);
  if (st != DIST_OK) {
    dist_decoder_destroy(d);
    return st;
  }
  *out = d;
  return DIST_OK;
}

dist_status dist_decoder_destroy(dist_decoder* d) {
  if (!d) return DIST_OK;
  for (void* p : d->allocations) cudaFree(p);
  delete d;
  return DIST_OK;
}

int dist_decoder_has_bf16(const dist_decoder* d) { return d && d->tc.ok ? 1 : 0; }

dist_status dist_decoder_device_error(const dist_decoder* d, int32_t* code) {
  DIST_CHECK(d && code, DIST_E_INVALID, "dist_decoder_device_error: NULL argument");
  *code = 0;
  if (!d->tc.ok) return DIST_OK;
  DIST_CUDA_TRY(cudaDeviceSynchronize());
  int v = 0;
  DIST_CUDA_TRY(cudaMemcpy(&v, d->tc.err, sizeof(int), cudaMemcpyDeviceToHost));
  DIST_CUDA_TRY(cudaMemset(d->tc.err, 0, sizeof(int)));
  *code = v;
  DIST_CHECK((v & 63) == 0, DIST_E_TIMEOUT,
             "a bounded wait of a tensor-core kernel ran out (outputs since the last check "
             "are invalid)");
  return DIST_OK;
}

dist_status dist_decoder_set_wait_limit(dist_decoder* d, uint64_t wait_ns, int withhold_copies) {
  DIST_CHECK(d, DIST_E_INVALID, "dist_decoder_set_wait_limit: NULL decoder");
  DIST_CHECK(d->tc.ok, DIST_E_UNSUPPORTED, "dist_decoder_set_wait_limit: no tensor-core path");
  DIST_CHECK(wait_ns >= 10000ull && wait_ns <= 10000000000ull, DIST_E_INVALID,
             "dist_decoder_set_wait_limit: wait_ns must be 1e4..1e10");
  d->tc.wait_ns = wait_ns;
  d->tc.withhold = withhold_copies != 0;
  return DIST_OK;
}

dist_status dist_workspace_create(int64_t max_rays, int max_steps, dist_workspace** out) {
  DIST_CHECK(out && max_rays > 0 && max_rays <= (int64_t)1 << 28 && max_steps > 0 &&
                 max_steps <= 100000,
             DIST_E_INVALID, "dist_workspace_create: bad size");
  dist_workspace* w = new dist_workspace();
  w->max_rays = max_rays;
  w->max_steps = max_steps;
  w->max_cams = 4096;
  auto& L = w->allocations;
  const size_t n = (size_t)max_rays;
  const size_t np = n * kProbesPerRay;
  dist_status s = DIST_OK;
  void* p = nullptr;
#define WS_ALLOC(field, bytes)                         \
  if (s == DIST_OK) {                                  \
    s = dev_alloc(L, &p, (bytes));                     \
    w->field = reinterpret_cast<decltype(w->field)>(p); \
  }
  WS_ALLOC(dir, n * sizeof(float4));
  WS_ALLOC(st, n * sizeof(float4));
  WS_ALLOC(fq, n * sizeof(int));
  WS_ALLOC(fprev, n * sizeof(float));
  WS_ALLOC(dprev, n * sizeof(float));
  WS_ALLOC(act[0][0], n * sizeof(int));
  WS_ALLOC(act[0][1], n * sizeof(int));
  WS_ALLOC(act[1][0], n * sizeof(int));
  WS_ALLOC(act[1][1], n * sizeof(int));
  WS_ALLOC(act[0][2], n * sizeof(int));
  WS_ALLOC(act[1][2], n * sizeof(int));
  WS_ALLOC(fbuf[0], n * sizeof(float));
  WS_ALLOC(fbuf[1], n * sizeof(float));
  WS_ALLOC(fbuf[2], n * sizeof(float));
  WS_ALLOC(counts, ((size_t)(max_steps + 2) * 3 + 2 * kMaxCoarseLevels) * sizeof(int));
  WS_ALLOC(rstat, n * sizeof(int));
  WS_ALLOC(chunk, ((n + 31) / 32) * sizeof(int));
  WS_ALLOC(cams, (size_t)w->max_cams * sizeof(CamDev));
  WS_ALLOC(bfold, (size_t)2 * kMaxShapes * 512 * sizeof(float));
  WS_ALLOC(gacc, (size_t)2 * kMaxShapes * 512 * sizeof(double));
  WS_ALLOC(probe_p, np * sizeof(float4));
  WS_ALLOC(probe_q, np * sizeof(float4));
  WS_ALLOC(probe_pix, np * sizeof(int));
  WS_ALLOC(probe_out, np * 4 * sizeof(float));
  WS_ALLOC(probe_count, 8 * sizeof(int));
  WS_ALLOC(red, 8 * sizeof(double));
  WS_ALLOC(ired, 8 * sizeof(int));
  WS_ALLOC(tc_scratch, (size_t)num_sms() * kTcAdjScratchPerCta);
  WS_ALLOC(wide_scratch, tc_wide_scratch_bytes());
#undef WS_ALLOC
  w->step_seq = 0;
  if (s == DIST_OK &&
      cudaMemset(tc_wide_seq_flag(w->wide_scratch), 0, sizeof(unsigned long long)) != cudaSuccess) {
    set_error("dist_workspace_create: cudaMemset failed");
    s = DIST_E_CUDA;
  }
  if (s != DIST_OK) {
    dist_workspace_destroy(w);
    return s;
  }
  *out = w;
  return DIST_OK;
}

dist_status dist_workspace_destroy(dist_workspace* w) {
  if (!w) return DIST_OK;
  cudaDeviceSynchronize();
  for (void* p : w->allocations) cudaFree(p);
  delete w;
  return DIST_OK;
}

}  // extern "C"
