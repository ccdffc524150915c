// Learned local-expansion correction (the paper has no counterpart): a
// multilayer perceptron maps the order-3 multipoles of a cell's 27 nearest
// cells to the difference between its order-p_high local expansion and its
// order-3 one, so that L2P at order p_high can run after an order-3 cell
// convolution.  The plain order-p_high evaluation is the network's training
// target and its fallback.
//
// Network: 432 -> 256 -> 256 -> 121 (128 rows stored), GELU, BF16 operands and
// FP32 accumulation on the tensor cores (mlp.cu), FP32 master parameters and
// Adam state.  Parameter layout (one flat FP32 vector):
//   W1 [256 x 432], b1 [256], W2 [256 x 256], b2 [256], W3 [128 x 256], b3 [128].
// Features are device-unit multipoles M' = M / hs^l times in_scale[channel];
// targets are device-unit locals L' = hs^(l+1) L times out_scale[channel].
#include <string.h>

#include <new>
#include <vector>

#include "plan.cuh"

using namespace pmmm;

namespace {

constexpr int S_IN = 432, S_H = 256, S_OP = 128, S_CLO = 16;
constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + (int64_t)S_H * S_IN, OFF_W2 = OFF_B1 + S_H,
                  OFF_B2 = OFF_W2 + (int64_t)S_H * S_H, OFF_W3 = OFF_B2 + S_H, OFF_B3 = OFF_W3 + (int64_t)S_OP * S_H,
                  NPARAM = OFF_B3 + S_OP;
constexpr int LOSS_PARTS = 512;
static_assert(NPARAM == PMMM_SUR_NPARAM, "parameter count");

}  // namespace

struct pmmm_surrogate {
  pmmm_plan* lo = nullptr;
  pmmm_plan* hi = nullptr;
  cudaStream_t stream = nullptr;
  int p_lo = 3, p_hi = 10, C_lo = S_CLO, C_hi = 121;
  int fallback = 0;
  int64_t step = 0;
  int64_t K = 0, Kp = 0;  // cells, cells rounded up to 128
  float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2t = nullptr, *W3t = nullptr;
  float *in_scale = nullptr, *out_scale = nullptr;
  bool stale = true;  // BF16 copies out of date
  int64_t cap = 0;
  __nv_bfloat16 *Y1 = nullptr, *Y2 = nullptr, *dO16 = nullptr, *dZ2_16 = nullptr, *dZ1_16 = nullptr;
  __nv_bfloat16 *Xt = nullptr, *Y1t = nullptr, *Y2t = nullptr, *dOt = nullptr, *dZ2t = nullptr, *dZ1t = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *O = nullptr, *dO = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  __nv_bfloat16* Xc = nullptr;  // features of the evaluated system [Kp][432]
  float* Lcorr = nullptr;       // corrected locals [C_hi][K]
  double *part = nullptr, *loss_d = nullptr, *stats_d = nullptr;
  int* err = nullptr;
  std::vector<void*> allocs;
  pmmm::FarHook hook;
};

namespace {

template <typename T>
cudaError_t salloc(pmmm_surrogate* s, T** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, sizeof(T) * (count ? count : 1));
  if (e == cudaSuccess) s->allocs.push_back(v);
  *p = (T*)v;
  return e;
}

void sfree(pmmm_surrogate* s, void* p) {
  if (!p) return;
  for (auto& a : s->allocs)
    if (a == p) {
      cudaFree(p);
      a = nullptr;
    }
}

int ensure_ws(pmmm_surrogate* s, int64_t rows) {
  if (rows <= s->cap) return PMMM_OK;
  cudaStreamSynchronize(s->stream);
  void* old[] = {s->Y1, s->Y2, s->dO16, s->dZ2_16, s->dZ1_16, s->Xt, s->Y1t, s->Y2t, s->dOt, s->dZ2t, s->dZ1t,
                 s->Z1, s->Z2, s->O, s->dO, s->dZ2, s->dZ1};
  for (void* p : old) sfree(s, p);
  s->cap = 0;
  cudaError_t e = cudaSuccess;
  const size_t R = (size_t)rows;
  if (e == cudaSuccess) e = salloc(s, &s->Y1, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->Y2, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->dO16, R * S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->dZ2_16, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->dZ1_16, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->Xt, R * S_IN);
  if (e == cudaSuccess) e = salloc(s, &s->Y1t, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->Y2t, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->dOt, R * S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->dZ2t, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->dZ1t, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->Z1, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->Z2, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->O, R * S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->dO, R * S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->dZ2, R * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->dZ1, R * S_H);
  if (e != cudaSuccess) return plan_map_cuda(e);
  s->cap = rows;
  return PMMM_OK;
}

#define SCK(x)                          \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

cudaError_t refresh_bf16(pmmm_surrogate* s, int* nl) {
  if (!s->stale) return cudaSuccess;
  cudaStream_t st = s->stream;
  SCK(launch_to_bf16(s->theta + OFF_W1, s->W1b, (int64_t)S_H * S_IN, st, nl));
  SCK(launch_to_bf16(s->theta + OFF_W2, s->W2b, (int64_t)S_H * S_H, st, nl));
  SCK(launch_to_bf16(s->theta + OFF_W3, s->W3b, (int64_t)S_OP * S_H, st, nl));
  SCK(launch_transpose_bf16(s->W2b, S_H, s->W2t, S_H, S_H, S_H, st, nl));    // W2t[i][o] = W2[o][i]
  SCK(launch_transpose_bf16(s->W3b, S_H, s->W3t, S_OP, S_OP, S_H, st, nl));  // W3t [256 x 128]
  s->stale = false;
  return cudaSuccess;
}

GemmArgs gemm(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* B, int64_t ldb, int M, int N, int K) {
  GemmArgs g;
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.M = M;
  g.N = N;
  g.K = K;
  return g;
}

// forward pass of `rows` feature rows X [rows][432] -> O [rows][128] (Z1, Y1, Z2, Y2 kept)
cudaError_t forward(pmmm_surrogate* s, const __nv_bfloat16* X, int rows, int* nl) {
  cudaStream_t st = s->stream;
  SCK(refresh_bf16(s, nl));
  GemmArgs g = gemm(X, S_IN, s->W1b, S_IN, rows, S_H, S_IN);
  g.bias = s->theta + OFF_B1;
  g.epi = GEMM_EPI_GELU;
  g.D32 = s->Z1;
  g.ldd = S_H;
  g.D16 = s->Y1;
  g.ldd16 = S_H;
  g.err = s->err;
  SCK(launch_gemm_tc(g, st, nl));
  g = gemm(s->Y1, S_H, s->W2b, S_H, rows, S_H, S_H);
  g.bias = s->theta + OFF_B2;
  g.epi = GEMM_EPI_GELU;
  g.D32 = s->Z2;
  g.ldd = S_H;
  g.D16 = s->Y2;
  g.ldd16 = S_H;
  g.err = s->err;
  SCK(launch_gemm_tc(g, st, nl));
  g = gemm(s->Y2, S_H, s->W3b, S_H, rows, S_OP, S_H);
  g.bias = s->theta + OFF_B3;
  g.D32 = s->O;
  g.ldd = S_OP;
  g.err = s->err;
  return launch_gemm_tc(g, st, nl);
}

// gradients of the mean-squared error of the last forward pass against T into s->grad
cudaError_t backward(pmmm_surrogate* s, const __nv_bfloat16* X, const float* T, int rows, int* nl) {
  cudaStream_t st = s->stream;
  SCK(launch_mse_grad(s->O, T, rows, S_OP, s->C_hi, s->dO, s->dO16, s->part, LOSS_PARTS, s->loss_d, st, nl));
  SCK(launch_colsum(s->dO, S_OP, rows, S_OP, s->grad + OFF_B3, st, nl));
  SCK(launch_transpose_bf16(s->dO16, S_OP, s->dOt, rows, rows, S_OP, st, nl));
  SCK(launch_transpose_bf16(s->Y2, S_H, s->Y2t, rows, rows, S_H, st, nl));
  GemmArgs g = gemm(s->dOt, rows, s->Y2t, rows, S_OP, S_H, rows);  // dW3 = dO^T Y2
  g.D32 = s->grad + OFF_W3;
  g.ldd = S_H;
  g.err = s->err;
  SCK(launch_gemm_tc(g, st, nl));
  g = gemm(s->dO16, S_OP, s->W3t, S_OP, rows, S_H, S_OP);  // dZ2 = (dO W3) * gelu'(Z2)
  g.epi = GEMM_EPI_DGELU;
  g.Zin = s->Z2;
  g.ldz = S_H;
  g.D32 = s->dZ2;
  g.ldd = S_H;
  g.D16 = s->dZ2_16;
  g.ldd16 = S_H;
  g.err = s->err;
  SCK(launch_gemm_tc(g, st, nl));
  SCK(launch_colsum(s->dZ2, S_H, rows, S_H, s->grad + OFF_B2, st, nl));
  SCK(launch_transpose_bf16(s->dZ2_16, S_H, s->dZ2t, rows, rows, S_H, st, nl));
  SCK(launch_transpose_bf16(s->Y1, S_H, s->Y1t, rows, rows, S_H, st, nl));
  g = gemm(s->dZ2t, rows, s->Y1t, rows, S_H, S_H, rows);  // dW2 = dZ2^T Y1
  g.D32 = s->grad + OFF_W2;
  g.ldd = S_H;
  g.err = s->err;
  SCK(launch_gemm_tc(g, st, nl));
  g = gemm(s->dZ2_16, S_H, s->W2t, S_H, rows, S_H, S_H);  // dZ1 = (dZ2 W2) * gelu'(Z1)
  g.epi = GEMM_EPI_DGELU;
  g.Zin = s->Z1;
  g.ldz = S_H;
  g.D32 = s->dZ1;
  g.ldd = S_H;
  g.D16 = s->dZ1_16;
  g.ldd16 = S_H;
  g.err = s->err;
  SCK(launch_gemm_tc(g, st, nl));
  SCK(launch_colsum(s->dZ1, S_H, rows, S_H, s->grad + OFF_B1, st, nl));
  SCK(launch_transpose_bf16(s->dZ1_16, S_H, s->dZ1t, rows, rows, S_H, st, nl));
  SCK(launch_transpose_bf16(X, S_IN, s->Xt, rows, rows, S_IN, st, nl));
  g = gemm(s->dZ1t, rows, s->Xt, rows, S_H, S_IN, rows);  // dW1 = dZ1^T X
  g.D32 = s->grad + OFF_W1;
  g.ldd = S_IN;
  g.err = s->err;
  return launch_gemm_tc(g, st, nl);
}

void free_sur(pmmm_surrogate* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void* p : s->allocs)
    if (p) cudaFree(p);
  s->allocs.clear();
  if (s->lo) pmmm_plan_destroy(s->lo);
  if (s->hi) pmmm_plan_destroy(s->hi);
}

int status_of(pmmm_surrogate* s, cudaError_t e) {
  if (e != cudaSuccess) return plan_map_cuda(e);
  int h = 0;
  e = cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return plan_map_cuda(e);
  if (h) {
    cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
    return PMMM_ERR_TIMEOUT;
  }
  return PMMM_OK;
}

bool rows_ok(int64_t rows) { return rows > 0 && rows % 128 == 0 && rows <= (int64_t)1 << 26; }

}  // namespace

extern "C" {

int pmmm_surrogate_create(const pmmm_config* cfg, int32_t p_high, void* stream, pmmm_surrogate** out) {
  if (!out || !cfg) return PMMM_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->p != 3 || p_high <= 3 || p_high > 10 || cfg->cutoff != 1) return PMMM_ERR_UNSUPPORTED;
  if (cfg->precision != PMMM_FP32 || cfg->refine > 1) return PMMM_ERR_UNSUPPORTED;
  pmmm_surrogate* s = new (std::nothrow) pmmm_surrogate();
  if (!s) return PMMM_ERR_OOM;
  s->stream = (cudaStream_t)stream;
  s->p_hi = p_high;
  s->C_hi = (p_high + 1) * (p_high + 1);
  pmmm_config chi = *cfg;
  chi.p = p_high;
  int rc = pmmm_plan_create(cfg, stream, &s->lo);
  if (rc == PMMM_OK) rc = pmmm_plan_create(&chi, stream, &s->hi);
  if (rc != PMMM_OK) {
    free_sur(s);
    delete s;
    return rc;
  }
  s->K = (int64_t)cfg->mesh[0] * cfg->mesh[1] * cfg->mesh[2];
  s->Kp = (s->K + 127) / 128 * 128;
  cudaError_t e = salloc(s, &s->theta, NPARAM);
  if (e == cudaSuccess) e = salloc(s, &s->grad, NPARAM);
  if (e == cudaSuccess) e = salloc(s, &s->am, NPARAM);
  if (e == cudaSuccess) e = salloc(s, &s->av, NPARAM);
  if (e == cudaSuccess) e = salloc(s, &s->W1b, (size_t)S_H * S_IN);
  if (e == cudaSuccess) e = salloc(s, &s->W2b, (size_t)S_H * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->W3b, (size_t)S_OP * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->W2t, (size_t)S_H * S_H);
  if (e == cudaSuccess) e = salloc(s, &s->W3t, (size_t)S_H * S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->in_scale, S_CLO);
  if (e == cudaSuccess) e = salloc(s, &s->out_scale, S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->Xc, (size_t)s->Kp * S_IN);
  if (e == cudaSuccess) e = salloc(s, &s->Lcorr, (size_t)s->C_hi * s->K);
  if (e == cudaSuccess) e = salloc(s, &s->part, LOSS_PARTS);
  if (e == cudaSuccess) e = salloc(s, &s->loss_d, 1);
  if (e == cudaSuccess) e = salloc(s, &s->stats_d, S_CLO + S_OP);
  if (e == cudaSuccess) e = salloc(s, &s->err, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->theta, 0, sizeof(float) * NPARAM, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->am, 0, sizeof(float) * NPARAM, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->av, 0, sizeof(float) * NPARAM, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->Xc, 0, sizeof(__nv_bfloat16) * (size_t)s->Kp * S_IN, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) {
    std::vector<float> ones(S_OP, 1.0f);
    e = cudaMemcpy(s->in_scale, ones.data(), sizeof(float) * S_CLO, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(s->out_scale, ones.data(), sizeof(float) * S_OP, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    rc = plan_map_cuda(e);
    free_sur(s);
    delete s;
    return rc;
  }
  *out = s;
  return PMMM_OK;
}

int pmmm_surrogate_destroy(pmmm_surrogate* s) {
  if (!s) return PMMM_OK;
  free_sur(s);
  delete s;
  return PMMM_OK;
}

static float* state_ptr(pmmm_surrogate* s, int what, int64_t* count) {
  switch (what) {
    case PMMM_SUR_PARAMS: *count = NPARAM; return s->theta;
    case PMMM_SUR_ADAM_M: *count = NPARAM; return s->am;
    case PMMM_SUR_ADAM_V: *count = NPARAM; return s->av;
    case PMMM_SUR_IN_SCALE: *count = S_CLO; return s->in_scale;
    case PMMM_SUR_OUT_SCALE: *count = s->C_hi; return s->out_scale;
    default: return nullptr;
  }
}

int pmmm_surrogate_get(pmmm_surrogate* s, int what, float* host, int64_t count) {
  if (!s || !host) return PMMM_ERR_INVALID_ARG;
  int64_t n = 0;
  float* p = state_ptr(s, what, &n);
  if (!p || count != n) return PMMM_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(host, p, sizeof(float) * n, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return plan_map_cuda(e);
}

int pmmm_surrogate_set(pmmm_surrogate* s, int what, const float* host, int64_t count) {
  if (!s || !host) return PMMM_ERR_INVALID_ARG;
  int64_t n = 0;
  float* p = state_ptr(s, what, &n);
  if (!p || count != n) return PMMM_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess) e = cudaMemcpy(p, host, sizeof(float) * n, cudaMemcpyHostToDevice);
  if (what == PMMM_SUR_PARAMS) s->stale = true;
  return plan_map_cuda(e);
}

int pmmm_surrogate_info(pmmm_surrogate* s, int what, int64_t* v) {
  if (!s || !v) return PMMM_ERR_INVALID_ARG;
  switch (what) {
    case PMMM_SUR_INFO_STEP: *v = s->step; break;
    case PMMM_SUR_INFO_FALLBACK: *v = s->fallback; break;
    case PMMM_SUR_INFO_CLOW: *v = s->C_lo; break;
    case PMMM_SUR_INFO_CHIGH: *v = s->C_hi; break;
    case PMMM_SUR_INFO_ROWS: *v = s->Kp; break;
    default: return PMMM_ERR_INVALID_ARG;
  }
  return PMMM_OK;
}

int pmmm_surrogate_set_step(pmmm_surrogate* s, int64_t step) {
  if (!s || step < 0) return PMMM_ERR_INVALID_ARG;
  s->step = step;
  return PMMM_OK;
}

int pmmm_surrogate_set_fallback(pmmm_surrogate* s, int on) {
  if (!s) return PMMM_ERR_INVALID_ARG;
  s->fallback = on ? 1 : 0;
  return PMMM_OK;
}

int pmmm_surrogate_training_pair(pmmm_surrogate* s, int64_t n, const void* pos, const void* q, void* X, float* T,
                                 double* stats) {
  if (!s || !X || !T || n < 0 || n > INT32_MAX || (n > 0 && (!pos || !q))) return PMMM_ERR_INVALID_ARG;
  int rc = plan_run(s->lo, 1, n, pos, q, nullptr, nullptr);
  if (rc == PMMM_OK) rc = plan_run(s->hi, 1, n, pos, q, nullptr, nullptr);
  if (rc != PMMM_OK) return rc;
  int nl = 0;
  cudaStream_t st = s->stream;
  const int nmesh[3] = {s->lo->cfg.mesh[0], s->lo->cfg.mesh[1], s->lo->cfg.mesh[2]};
  cudaError_t e = cudaSuccess;
  if (s->Kp > s->K)
    e = cudaMemsetAsync((__nv_bfloat16*)X + s->K * S_IN, 0, sizeof(__nv_bfloat16) * (size_t)(s->Kp - s->K) * S_IN, st);
  if (e == cudaSuccess)
    e = launch_gather_features((const float*)s->lo->M, s->K, nmesh, s->lo->g.periodic, s->in_scale, X, S_IN, st, &nl);
  if (e == cudaSuccess && s->Kp > s->K)
    e = cudaMemsetAsync(T + s->K * S_OP, 0, sizeof(float) * (size_t)(s->Kp - s->K) * S_OP, st);
  if (e == cudaSuccess)
    e = launch_build_targets((const float*)s->hi->L, (const float*)s->lo->L, s->K, s->C_hi, s->C_lo, s->out_scale, T,
                             S_OP, st, &nl);
  if (e == cudaSuccess && stats) {
    e = cudaMemsetAsync(s->stats_d, 0, sizeof(double) * (S_CLO + S_OP), st);
    if (e == cudaSuccess) e = launch_channel_sumsq((const float*)s->lo->M, S_CLO, s->K, s->stats_d, st, &nl);
    if (e == cudaSuccess)
      e = launch_diff_sumsq((const float*)s->hi->L, (const float*)s->lo->L, s->C_hi, s->C_lo, s->K, s->stats_d + S_CLO,
                            st, &nl);
    std::vector<double> h(S_CLO + S_OP);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data(), s->stats_d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
      for (int c = 0; c < S_CLO + s->C_hi; ++c) stats[c] += h[c];
  }
  return status_of(s, e);
}

int pmmm_surrogate_forward(pmmm_surrogate* s, const void* X, int64_t rows, float* out) {
  if (!s || !X || !out || !rows_ok(rows)) return PMMM_ERR_INVALID_ARG;
  int rc = ensure_ws(s, rows);
  if (rc != PMMM_OK) return rc;
  int nl = 0;
  cudaError_t e = forward(s, (const __nv_bfloat16*)X, (int)rows, &nl);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, s->O, sizeof(float) * (size_t)rows * S_OP, cudaMemcpyDeviceToDevice, s->stream);
  return status_of(s, e);
}

int pmmm_surrogate_gradients(pmmm_surrogate* s, const void* X, const float* T, int64_t rows, float* grad_host,
                             double* loss) {
  if (!s || !X || !T || !rows_ok(rows)) return PMMM_ERR_INVALID_ARG;
  int rc = ensure_ws(s, rows);
  if (rc != PMMM_OK) return rc;
  int nl = 0;
  cudaError_t e = forward(s, (const __nv_bfloat16*)X, (int)rows, &nl);
  if (e == cudaSuccess) e = backward(s, (const __nv_bfloat16*)X, T, (int)rows, &nl);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, s->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, s->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  return status_of(s, e);
}

int pmmm_surrogate_train_step(pmmm_surrogate* s, const void* X, const float* T, int64_t rows, float lr, double* loss) {
  if (!s || !X || !T || !rows_ok(rows) || !(lr > 0.f)) return PMMM_ERR_INVALID_ARG;
  int rc = ensure_ws(s, rows);
  if (rc != PMMM_OK) return rc;
  int nl = 0;
  cudaError_t e = forward(s, (const __nv_bfloat16*)X, (int)rows, &nl);
  if (e == cudaSuccess) e = backward(s, (const __nv_bfloat16*)X, T, (int)rows, &nl);
  if (e == cudaSuccess) e = launch_adam(s->theta, s->grad, s->am, s->av, NPARAM, lr, s->step + 1, s->stream, &nl);
  if (e != cudaSuccess) return plan_map_cuda(e);
  s->step += 1;
  s->stale = true;
  if (!loss) return PMMM_OK;
  e = cudaMemcpyAsync(loss, s->loss_d, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  return status_of(s, e);
}

int pmmm_surrogate_compute(pmmm_surrogate* s, int64_t n, const void* pos, const void* q, void* phi, void* force,
                           double* energy) {
  if (!s || n < 0 || n > INT32_MAX || (n > 0 && (!pos || !q))) return PMMM_ERR_INVALID_ARG;
  if (s->fallback) return pmmm_compute(s->hi, n, pos, q, phi, force, energy);
  int rc = ensure_ws(s, s->Kp);
  if (rc != PMMM_OK) return rc;
  const int nmesh[3] = {s->lo->cfg.mesh[0], s->lo->cfg.mesh[1], s->lo->cfg.mesh[2]};
  s->hook.fn = [s, nmesh](cudaStream_t st, int* nl) -> cudaError_t {
    SCK(launch_gather_features((const float*)s->lo->M, s->K, nmesh, s->lo->g.periodic, s->in_scale, s->Xc, S_IN, st,
                               nl));
    SCK(forward(s, s->Xc, (int)s->Kp, nl));
    return launch_combine_locals((const float*)s->lo->L, s->O, S_OP, s->K, s->C_hi, s->C_lo, s->out_scale, s->Lcorr,
                                 st, nl);
  };
  s->hook.p_l2p = s->p_hi;
  s->hook.L = s->Lcorr;
  s->lo->hook = &s->hook;
  rc = plan_run(s->lo, 1, n, pos, q, phi, force);
  s->lo->hook = nullptr;
  if (rc != PMMM_OK) return rc;
  if (!energy) return PMMM_OK;
  rc = plan_read_energies(s->lo, 1, energy);
  if (rc != PMMM_OK) return rc;
  return status_of(s, cudaSuccess);
}

}  // extern "C"
