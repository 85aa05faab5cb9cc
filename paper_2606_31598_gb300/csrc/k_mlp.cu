// k_mlp.cu -- the learned plan-selection surrogate (Sec. IV.C, Algorithm 3):
// a multilayer perceptron f(x) = tanh(tanh(z W1 + b1) W2 + b2) W3 + b3 on
// the z-scored feature vector z = (x - mu)/sigma (Eq. nn_surrogate with one
// more hidden layer), trained on the log of measured times with a masked
// mean-squared error (Eq. nn_loss), one output per storage strategy
// (procedural, partial, full).  Forward, backward and Adam run in the
// kernels below (FP32); every reduction over samples runs in index order, so
// training is deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mf_internal.h"

struct mf_mlp {
  int F = 0, H = 0, O = 0;
  int64_t nparams = 0;
  float* d_par = nullptr;
  float* d_grad = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  std::vector<float> mu, sd;
  int64_t adam_t = 0;
  // per-batch buffers
  int64_t ncap = 0;
  float *d_x = nullptr, *d_y = nullptr, *d_mask = nullptr, *d_z0 = nullptr, *d_a1 = nullptr, *d_a2 = nullptr,
        *d_out = nullptr, *d_g2 = nullptr, *d_g1 = nullptr, *d_g0 = nullptr, *d_norm = nullptr, *d_loss = nullptr;
};

namespace mf {
namespace {

inline unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1 << 16)); }

// z = (x - mu) / sd, row-major [n][F]
__global__ void k_norm(const float* __restrict__ x, const float* __restrict__ musd, float* __restrict__ z, int64_t n,
                       int F) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * F; e += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(e % F);
    z[e] = (x[e] - musd[f]) / musd[F + f];
  }
}

// out[i][o] = act(b[o] + sum_k in[i][k] W[k][o])
__global__ void k_dense(const float* __restrict__ in, const float* __restrict__ W, const float* __restrict__ b,
                        float* __restrict__ out, int64_t n, int fin, int fout, int act_tanh) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * fout; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / fout;
    const int o = (int)(e % fout);
    float s = b[o];
    for (int k = 0; k < fin; ++k) s = fmaf(in[i * fin + k], W[k * fout + o], s);
    out[e] = act_tanh ? tanhf(s) : s;
  }
}

// g_out[i][o] = 2 mask (out - y) / nmask
__global__ void k_out_grad(const float* __restrict__ out, const float* __restrict__ y, const float* __restrict__ mask,
                           float* __restrict__ g, int64_t n, int O, float inv_nmask) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * O; e += (int64_t)gridDim.x * blockDim.x)
    g[e] = 2.0f * mask[e] * (out[e] - y[e]) * inv_nmask;
}

// loss = sum mask (out - y)^2 / nmask; one CTA, index-ordered partials
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ y, const float* __restrict__ mask,
                       int64_t m, float inv_nmask, float* __restrict__ loss) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < m; e += 256) {
    const double d = (double)out[e] - (double)y[e];
    s += (double)mask[e] * d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(sh[0] * inv_nmask);
}

// dW[k][o] = sum_i in[i][k] g[i][o];  db[o] = sum_i g[i][o]   (i in order)
__global__ void k_grad_w(const float* __restrict__ in, const float* __restrict__ g, float* __restrict__ dW,
                         float* __restrict__ db, int64_t n, int fin, int fout) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < (int64_t)fin * fout) {
    const int k = (int)(e / fout), o = (int)(e % fout);
    float s = 0.f;
    for (int64_t i = 0; i < n; ++i) s = fmaf(in[i * fin + k], g[i * fout + o], s);
    dW[e] = s;
  } else if (e < (int64_t)fin * fout + fout) {
    const int o = (int)(e - (int64_t)fin * fout);
    float s = 0.f;
    for (int64_t i = 0; i < n; ++i) s += g[i * fout + o];
    db[o] = s;
  }
}

// gin[i][k] = (sum_o g[i][o] W[k][o]) * (1 - a[i][k]^2)    (back through tanh)
__global__ void k_back(const float* __restrict__ g, const float* __restrict__ W, const float* __restrict__ a,
                       float* __restrict__ gin, int64_t n, int fin, int fout) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * fin; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / fin;
    const int k = (int)(e % fin);
    float s = 0.f;
    for (int o = 0; o < fout; ++o) s = fmaf(g[i * fout + o], W[k * fout + o], s);
    const float av = a[e];
    gin[e] = s * (1.0f - av * av);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

template <typename T>
void freep(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

struct Offsets {
  int64_t W1, b1, W2, b2, W3, b3, n;
};
Offsets offsets(const mf_mlp& m) {
  Offsets o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)m.F * m.H;
  o.W2 = o.b1 + m.H;
  o.b2 = o.W2 + (int64_t)m.H * m.H;
  o.W3 = o.b2 + m.H;
  o.b3 = o.W3 + (int64_t)m.H * m.O;
  o.n = o.b3 + m.O;
  return o;
}

mf_status ensure_batch(mf_mlp& m, int64_t n) {
  if (n <= m.ncap) return MF_OK;
  float** bufs[] = {&m.d_x, &m.d_y, &m.d_mask, &m.d_z0, &m.d_a1, &m.d_a2, &m.d_out, &m.d_g2, &m.d_g1, &m.d_g0};
  for (auto b : bufs) freep(*b);
  const int W = std::max(m.F, std::max(m.H, m.O));
  for (auto b : bufs)
    if (cudaMalloc((void**)b, (size_t)n * W * sizeof(float)) != cudaSuccess) return MF_ERR_OOM;
  m.ncap = n;
  return MF_OK;
}

// forward of n samples already in d_x: z0, a1, a2, out
cudaError_t forward(mf_mlp& m, int64_t n) {
  const Offsets o = offsets(m);
  k_norm<<<blocks_for(n * m.F), 256>>>(m.d_x, m.d_norm, m.d_z0, n, m.F);
  k_dense<<<blocks_for(n * m.H), 256>>>(m.d_z0, m.d_par + o.W1, m.d_par + o.b1, m.d_a1, n, m.F, m.H, 1);
  k_dense<<<blocks_for(n * m.H), 256>>>(m.d_a1, m.d_par + o.W2, m.d_par + o.b2, m.d_a2, n, m.H, m.H, 1);
  k_dense<<<blocks_for(n * m.O), 256>>>(m.d_a2, m.d_par + o.W3, m.d_par + o.b3, m.d_out, n, m.H, m.O, 0);
  return cudaGetLastError();
}

// loss and gradient of the masked MSE for the batch in d_x/d_y/d_mask
cudaError_t loss_grad(mf_mlp& m, int64_t n, float inv_nmask) {
  const Offsets o = offsets(m);
  cudaError_t e = forward(m, n);
  if (e != cudaSuccess) return e;
  k_loss<<<1, 256>>>(m.d_out, m.d_y, m.d_mask, n * m.O, inv_nmask, m.d_loss);
  k_out_grad<<<blocks_for(n * m.O), 256>>>(m.d_out, m.d_y, m.d_mask, m.d_g2, n, m.O, inv_nmask);
  k_grad_w<<<blocks_for((int64_t)m.H * m.O + m.O), 256>>>(m.d_a2, m.d_g2, m.d_grad + o.W3, m.d_grad + o.b3, n, m.H,
                                                           m.O);
  k_back<<<blocks_for(n * m.H), 256>>>(m.d_g2, m.d_par + o.W3, m.d_a2, m.d_g1, n, m.H, m.O);
  k_grad_w<<<blocks_for((int64_t)m.H * m.H + m.H), 256>>>(m.d_a1, m.d_g1, m.d_grad + o.W2, m.d_grad + o.b2, n, m.H,
                                                           m.H);
  k_back<<<blocks_for(n * m.H), 256>>>(m.d_g1, m.d_par + o.W2, m.d_a1, m.d_g0, n, m.H, m.H);
  k_grad_w<<<blocks_for((int64_t)m.F * m.H + m.H), 256>>>(m.d_z0, m.d_g0, m.d_grad + o.W1, m.d_grad + o.b1, n, m.F,
                                                           m.H);
  return cudaGetLastError();
}

mf_status upload_batch(mf_mlp& m, const float* X, const float* Y, const float* mask, int64_t n, float* inv_nmask) {
  mf_status st = ensure_batch(m, n);
  if (st != MF_OK) return st;
  if (cudaMemcpy(m.d_x, X, (size_t)n * m.F * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MF_ERR_CUDA;
  if (Y && cudaMemcpy(m.d_y, Y, (size_t)n * m.O * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return MF_ERR_CUDA;
  if (Y) {
    std::vector<float> mk((size_t)n * m.O, 1.0f);
    if (mask) std::memcpy(mk.data(), mask, mk.size() * sizeof(float));
    double cnt = 0;
    for (float v : mk) cnt += v;
    if (cnt <= 0) return MF_ERR_INVALID;
    if (inv_nmask) *inv_nmask = (float)(1.0 / cnt);
    if (cudaMemcpy(m.d_mask, mk.data(), mk.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return MF_ERR_CUDA;
  }
  return MF_OK;
}

mf_status upload_norm(mf_mlp& m) {
  std::vector<float> ms(m.mu);
  ms.insert(ms.end(), m.sd.begin(), m.sd.end());
  return cudaMemcpy(m.d_norm, ms.data(), ms.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess
             ? MF_OK
             : MF_ERR_CUDA;
}

// splitmix64 -> uniform(-1, 1), for the Glorot-uniform initial weights
double unif(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return ((double)(z >> 11) + 0.5) * 0x1p-53 * 2.0 - 1.0;
}

}  // namespace

// Feature vector of a candidate plan for the surrogate (10 entries).
void mlp_features(int32_t generator, int32_t precision, const mf_problem& pr, const mf_candidate& c,
                  const mf_estimate& e, double budget, float* x) {
  const double full_bytes = (double)e.n_pair * e.M_block;
  x[0] = (float)std::log2((double)pr.D_in);
  x[1] = (float)std::log2((double)(c.block > 0 ? c.block : pr.D_in));
  x[2] = (float)std::log2((double)pr.R);
  x[3] = precision == MF_PREC_FP32 ? 1.f : 0.f;
  x[4] = precision == MF_PREC_BF16X2 ? 1.f : 0.f;
  x[5] = precision == MF_PREC_FP64 ? 1.f : 0.f;
  x[6] = generator == MF_GEN_PHILOX_GUE ? 1.f : 0.f;
  x[7] = generator == MF_GEN_SINC_DVR_HO ? 1.f : 0.f;
  x[8] = (float)(full_bytes > 0 ? std::min(1.0, budget / full_bytes) : 1.0);
  x[9] = (float)std::log10(1.0 + budget / 1e9);
}

// Two surrogate forms.  Direct (10 inputs): the head of the candidate's
// storage mode predicts ln t_mv.  Residual (11 inputs): the eleventh input is
// ln of the analytic per-application time S_model / waves (Eq.
// planner_cost_score over Eq. planner_waves), and the head predicts the
// residual ln t_mv - ln(S_model / waves), so the network learns only where
// the runtime model misses.
mf_status surrogate_predict(void* model, int32_t generator, int32_t precision, const mf_problem& pr,
                            const mf_candidate& c, const mf_estimate& e, double budget, double, int, double* t) {
  mf_mlp* m = (mf_mlp*)model;
  if (!m || (m->F != 10 && m->F != 11) || m->O != 3) return MF_ERR_INVALID;
  float x[11], y[3];
  mlp_features(generator, precision, pr, c, e, budget, x);
  const double t_model = e.S_model / (double)std::max<int64_t>(1, e.waves);
  if (m->F == 11) {
    if (!(t_model > 0)) return MF_ERR_INVALID;
    x[10] = (float)std::log(t_model);
  }
  mf_status st = mf_mlp_predict(m, x, 1, y);
  if (st != MF_OK) return st;
  const int k = c.storage == MF_STORE_PROCEDURAL ? 0 : (c.storage == MF_STORE_PARTIAL ? 1 : 2);
  *t = std::exp((double)y[k]) * (m->F == 11 ? t_model : 1.0);
  return MF_OK;
}

}  // namespace mf

using namespace mf;

extern "C" {

mf_status mf_mlp_create(mf_mlp_t* out, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
    return MF_ERR_INVALID;
  *out = nullptr;
  mf_mlp* m = new (std::nothrow) mf_mlp();
  if (!m) return MF_ERR_OOM;
  m->F = n_in;
  m->H = n_hidden;
  m->O = n_out;
  const Offsets o = offsets(*m);
  m->nparams = o.n;
  m->mu.assign(n_in, 0.f);
  m->sd.assign(n_in, 1.f);
  float** bufs[] = {&m->d_par, &m->d_grad, &m->d_m, &m->d_v};
  for (auto b : bufs)
    if (cudaMalloc((void**)b, (size_t)o.n * sizeof(float)) != cudaSuccess) {
      mf_mlp_destroy(m);
      return MF_ERR_OOM;
    }
  if (cudaMalloc((void**)&m->d_norm, 2 * (size_t)n_in * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&m->d_loss, sizeof(float)) != cudaSuccess) {
    mf_mlp_destroy(m);
    return MF_ERR_OOM;
  }
  // Glorot-uniform weights, zero biases
  std::vector<float> par((size_t)o.n, 0.f);
  uint64_t s = seed;
  auto fill = [&](int64_t off, int fin, int fout) {
    const double a = std::sqrt(6.0 / (fin + fout));
    for (int64_t i = 0; i < (int64_t)fin * fout; ++i) par[(size_t)(off + i)] = (float)(a * unif(s));
  };
  fill(o.W1, n_in, n_hidden);
  fill(o.W2, n_hidden, n_hidden);
  fill(o.W3, n_hidden, n_out);
  if (cudaMemcpy(m->d_par, par.data(), par.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->d_m, 0, par.size() * sizeof(float)) != cudaSuccess ||
      cudaMemset(m->d_v, 0, par.size() * sizeof(float)) != cudaSuccess || upload_norm(*m) != MF_OK) {
    mf_mlp_destroy(m);
    return MF_ERR_CUDA;
  }
  *out = m;
  return MF_OK;
}

mf_status mf_mlp_destroy(mf_mlp_t m) {
  if (!m) return MF_OK;
  float** bufs[] = {&m->d_par, &m->d_grad, &m->d_m, &m->d_v, &m->d_x, &m->d_y, &m->d_mask, &m->d_z0, &m->d_a1,
                    &m->d_a2, &m->d_out, &m->d_g2, &m->d_g1, &m->d_g0, &m->d_norm, &m->d_loss};
  for (auto b : bufs) freep(*b);
  delete m;
  return MF_OK;
}

mf_status mf_mlp_param_count(mf_mlp_t m, int64_t* n) {
  if (!m || !n) return MF_ERR_INVALID;
  *n = m->nparams;
  return MF_OK;
}

mf_status mf_mlp_get_params(mf_mlp_t m, float* params, float* mu, float* sd) {
  if (!m) return MF_ERR_INVALID;
  if (params && cudaMemcpy(params, m->d_par, (size_t)m->nparams * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MF_ERR_CUDA;
  if (mu) std::memcpy(mu, m->mu.data(), m->mu.size() * sizeof(float));
  if (sd) std::memcpy(sd, m->sd.data(), m->sd.size() * sizeof(float));
  return MF_OK;
}

mf_status mf_mlp_set_params(mf_mlp_t m, const float* params, const float* mu, const float* sd) {
  if (!m) return MF_ERR_INVALID;
  if (params && cudaMemcpy(m->d_par, params, (size_t)m->nparams * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return MF_ERR_CUDA;
  if (mu) std::memcpy(m->mu.data(), mu, m->mu.size() * sizeof(float));
  if (sd)
    for (int f = 0; f < m->F; ++f) {
      if (!(sd[f] > 0)) return MF_ERR_INVALID;
      m->sd[f] = sd[f];
    }
  return upload_norm(*m);
}

mf_status mf_mlp_predict(mf_mlp_t m, const float* X, int64_t n, float* Y) {
  if (!m || !X || !Y || n < 1) return MF_ERR_INVALID;
  mf_status st = upload_batch(*m, X, nullptr, nullptr, n, nullptr);
  if (st != MF_OK) return st;
  if (forward(*m, n) != cudaSuccess) return MF_ERR_CUDA;
  if (cudaMemcpy(Y, m->d_out, (size_t)n * m->O * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MF_ERR_CUDA;
  return MF_OK;
}

mf_status mf_mlp_loss_grad(mf_mlp_t m, const float* X, const float* Y, const float* mask, int64_t n, float* loss,
                           float* grad) {
  if (!m || !X || !Y || n < 1) return MF_ERR_INVALID;
  float inv = 0.f;
  mf_status st = upload_batch(*m, X, Y, mask, n, &inv);
  if (st != MF_OK) return st;
  if (loss_grad(*m, n, inv) != cudaSuccess) return MF_ERR_CUDA;
  if (loss && cudaMemcpy(loss, m->d_loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MF_ERR_CUDA;
  if (grad && cudaMemcpy(grad, m->d_grad, (size_t)m->nparams * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MF_ERR_CUDA;
  return MF_OK;
}

mf_status mf_mlp_train(mf_mlp_t m, const float* X, const float* Y, const float* mask, int64_t n, int32_t epochs,
                       float lr, int32_t set_normalization, float* loss_curve) {
  if (!m || !X || !Y || n < 1 || epochs < 0 || !(lr > 0)) return MF_ERR_INVALID;
  if (set_normalization) {
    // z-score statistics of the training features (Sec. IV.C)
    for (int f = 0; f < m->F; ++f) {
      double s = 0, s2 = 0;
      for (int64_t i = 0; i < n; ++i) {
        const double v = X[i * m->F + f];
        s += v;
        s2 += v * v;
      }
      const double mu = s / n, var = std::max(0.0, s2 / n - mu * mu);
      m->mu[f] = (float)mu;
      m->sd[f] = (float)(var > 1e-12 ? std::sqrt(var) : 1.0);
    }
    mf_status st = upload_norm(*m);
    if (st != MF_OK) return st;
  }
  float inv = 0.f;
  mf_status st = upload_batch(*m, X, Y, mask, n, &inv);
  if (st != MF_OK) return st;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int32_t ep = 0; ep < epochs; ++ep) {
    if (loss_grad(*m, n, inv) != cudaSuccess) return MF_ERR_CUDA;
    if (loss_curve && cudaMemcpy(&loss_curve[ep], m->d_loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      return MF_ERR_CUDA;
    ++m->adam_t;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    k_adam<<<blocks_for(m->nparams), 256>>>(m->d_par, m->d_grad, m->d_m, m->d_v, m->nparams, lr, b1, b2, eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return MF_ERR_CUDA;
  return MF_OK;
}

mf_status mf_mlp_features(int32_t generator, int32_t precision, int64_t D, int64_t block, int64_t nvec,
                          double cache_budget_bytes, float* out10) {
  if (!out10 || D < 2 || nvec < 1 || block < 0) return MF_ERR_INVALID;
  const double eb = precision == MF_PREC_FP64 ? 16.0 : 8.0;
  mf_problem pr{D, D, nvec, 1, 1, eb, 1e12, 1};
  mf_candidate c{block, MF_STORE_PARTIAL, -1, 1, 1, 4};
  mf_estimate e{};
  planner_estimate(pr, c, mf_device_model{}, 0.9, cache_budget_bytes, e);
  mlp_features(generator, precision, pr, c, e, cache_budget_bytes, out10);
  return MF_OK;
}

}  // extern "C"
