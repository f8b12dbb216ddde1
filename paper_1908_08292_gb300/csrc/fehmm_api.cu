// C ABI of the batched FE-HMM RVE engine (declarations and contracts in include/fehmm.h).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <new>
#include <string>
#include <vector>

#include "fehmm.h"
#include "fehmm_device.cuh"
#include "rve_args.h"

using namespace fehmm;

struct fehmm_ctx {
  fehmm_options opt;
  int device = 0, num_sms = 0;
  // microstructures (host copies; device copies rebuilt on bind)
  std::vector<int32_t> rve_n;
  std::vector<int64_t> rve_phase_off;
  std::vector<uint8_t> phase;
  std::vector<double> lame;  // [n_rve][kMaxPhase][2]
  int32_t* d_rve_n = nullptr;
  int64_t* d_rve_phase_off = nullptr;
  uint8_t* d_phase = nullptr;
  double* d_lame = nullptr;
  // quadrature points
  int n_qp = 0, nn_max = 0;
  size_t w_total = 0;
  std::vector<int64_t> w_off_h;
  int32_t* d_qp_rve = nullptr;
  int32_t* d_order = nullptr;
  int64_t* d_w_off = nullptr;
  double* d_w_cur = nullptr;
  double* d_w_comm = nullptr;
  void* d_x_cur = nullptr;  // kept tangent-transfer solutions (fehmm_options.transfer_warm)
  void* d_x_comm = nullptr;
  size_t x_bytes = 0;
  int32_t* d_queue = nullptr;
  void* d_scratch = nullptr;
  size_t scratch_bytes = 0;
  // macro mesh
  bool has_macro = false;
  MacroArgs macro{};
  int32_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  int32_t* d_blk_base = nullptr;
  int32_t* d_blk_stride = nullptr;
  int macro_rows = 0, macro_nnz = 0;
  uint8_t* d_fixed = nullptr;   // Dirichlet mask of the macro dofs
  int32_t* d_fixed_dofs = nullptr;
  double* d_fixed_vals = nullptr;
  double* d_dir_full = nullptr;  // [macro_rows]: the Dirichlet end values on their dofs, 0 elsewhere
  int n_fixed = 0;
  double* d_solve_work = nullptr;
  long long launches = 0;
};

namespace {

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

template <typename T>
int dupload(T*& dst, const T* src, size_t count) {
  dfree(dst);
  if (count == 0) return FEHMM_OK;
  if (cudaMalloc((void**)&dst, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    dst = nullptr;
    return FEHMM_ERR_OOM;
  }
  if (cudaMemcpy(dst, src, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess) return FEHMM_ERR_CUDA;
  return FEHMM_OK;
}

bool valid_options(const fehmm_options* o) {
  return o && (o->dim == 2 || o->dim == 3) && (o->precision == FEHMM_PREC_FP64 || o->precision == FEHMM_PREC_MIXED) &&
         o->newton_rtol >= 0 && o->newton_atol >= 0 && o->max_newton >= 0 && o->cg_rtol > 0 && o->max_cg > 0 &&
         o->cond_rtol > 0 && o->max_cond_cg > 0 && o->retry_stages >= 0 && o->retry_stages <= 64 &&
         (o->precond == FEHMM_PRECOND_BLOCK_JACOBI || o->precond == FEHMM_PRECOND_MULTIGRID) &&
         (o->bc == FEHMM_BC_PERIODIC || o->bc == FEHMM_BC_KUBC) &&
         (o->law == FEHMM_LAW_NEO_HOOKE || o->law == FEHMM_LAW_SVK) && o->mg_omega > 0.0 && o->mg_omega < 1.0 &&
         (o->mg_reuse == 0 || o->mg_reuse == 1) && (o->transfer_warm == 0 || o->transfer_warm == 1);
}

}  // namespace

extern "C" {

int fehmm_default_options(fehmm_options* opt, int dim, int precision) {
  if (!opt || (dim != 2 && dim != 3) || (precision != FEHMM_PREC_FP64 && precision != FEHMM_PREC_MIXED))
    return FEHMM_ERR_ARG;
  opt->dim = dim;
  opt->precision = precision;
  opt->newton_rtol = 1e-10;
  opt->newton_atol = 1e-14;
  opt->max_newton = 25;
  opt->cg_rtol = precision == FEHMM_PREC_FP64 ? 1e-6 : 1e-4;
  opt->max_cg = 2000;
  opt->cond_rtol = precision == FEHMM_PREC_FP64 ? 1e-9 : 1e-6;
  opt->max_cond_cg = 4000;
  opt->retry_stages = 4;
  opt->precond = FEHMM_PRECOND_MULTIGRID;
  opt->bc = FEHMM_BC_PERIODIC;
  opt->law = FEHMM_LAW_NEO_HOOKE;
  opt->mg_omega = dim == 2 ? 0.7 : 0.6;
  opt->mg_reuse = 1;
  opt->transfer_warm = 1;
  return FEHMM_OK;
}

int fehmm_create(fehmm_ctx** out, const fehmm_options* opt) {
  if (!out || !valid_options(opt)) return FEHMM_ERR_ARG;
  *out = nullptr;
  fehmm_ctx* c = new (std::nothrow) fehmm_ctx();
  if (!c) return FEHMM_ERR_OOM;
  c->opt = *opt;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return FEHMM_ERR_CUDA;
  }
  if (cudaMalloc((void**)&c->d_queue, sizeof(int32_t) * 4) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return FEHMM_ERR_OOM;
  }
  *out = c;
  return FEHMM_OK;
}

int fehmm_destroy(fehmm_ctx* c) {
  if (!c) return FEHMM_ERR_ARG;
  dfree(c->d_rve_n);
  dfree(c->d_rve_phase_off);
  dfree(c->d_phase);
  dfree(c->d_lame);
  dfree(c->d_qp_rve);
  dfree(c->d_order);
  dfree(c->d_w_off);
  dfree(c->d_w_cur);
  dfree(c->d_w_comm);
  if (c->d_x_cur) cudaFree(c->d_x_cur);
  if (c->d_x_comm) cudaFree(c->d_x_comm);
  dfree(c->d_queue);
  if (c->d_scratch) cudaFree(c->d_scratch);
  dfree(c->d_rowptr);
  dfree(c->d_col);
  dfree(c->d_blk_base);
  dfree(c->d_blk_stride);
  dfree(c->d_fixed);
  dfree(c->d_fixed_dofs);
  dfree(c->d_fixed_vals);
  dfree(c->d_dir_full);
  dfree(c->d_solve_work);
  delete c;
  return FEHMM_OK;
}

int fehmm_get_options(const fehmm_ctx* c, fehmm_options* opt) {
  if (!c || !opt) return FEHMM_ERR_ARG;
  *opt = c->opt;
  return FEHMM_OK;
}

int fehmm_set_options(fehmm_ctx* c, const fehmm_options* opt) {
  if (!c || !valid_options(opt) || opt->dim != c->opt.dim || opt->precision != c->opt.precision) return FEHMM_ERR_ARG;
  c->opt = *opt;
  return FEHMM_OK;
}

int fehmm_add_rves(fehmm_ctx* c, int n_rve, const int32_t* grid_n, const uint8_t* phase, const double* E,
                   const double* nu, int n_phase, int* first_id) {
  if (!c || n_rve <= 0 || !grid_n || !phase || !E || !nu || n_phase <= 0 || n_phase > kMaxPhase) return FEHMM_ERR_ARG;
  const int d = c->opt.dim;
  for (int r = 0; r < n_rve; ++r) {
    const int n = grid_n[r];
    if (d == 2 && (n < 2 || n > 32)) return FEHMM_ERR_ARG;
    if (d == 2 && (n % 2) != 0) return FEHMM_ERR_UNSUPPORTED;
    if (d == 3 && (n < 2 || n > 16)) return FEHMM_ERR_ARG;
    for (int p = 0; p < n_phase; ++p) {
      const double e = E[(size_t)r * n_phase + p], v = nu[(size_t)r * n_phase + p];
      if (!(e > 0) || !(v > -1.0 && v < 0.5)) return FEHMM_ERR_ARG;
    }
  }
  // validate phase ids before touching the context
  size_t off = 0;
  for (int r = 0; r < n_rve; ++r) {
    size_t cnt = 1;
    for (int k = 0; k < d; ++k) cnt *= (size_t)grid_n[r];
    for (size_t i = 0; i < cnt; ++i)
      if (phase[off + i] >= n_phase) return FEHMM_ERR_ARG;
    off += cnt;
  }
  if (first_id) *first_id = (int)c->rve_n.size();
  off = 0;
  for (int r = 0; r < n_rve; ++r) {
    size_t cnt = 1;
    for (int k = 0; k < d; ++k) cnt *= (size_t)grid_n[r];
    c->rve_n.push_back(grid_n[r]);
    c->rve_phase_off.push_back((int64_t)c->phase.size());
    c->phase.insert(c->phase.end(), phase + off, phase + off + cnt);
    off += cnt;
    for (int p = 0; p < kMaxPhase; ++p) {
      double lam = 0, mu = 0;
      if (p < n_phase) lame_from_E_nu(E[(size_t)r * n_phase + p], nu[(size_t)r * n_phase + p], lam, mu);
      c->lame.push_back(lam);
      c->lame.push_back(mu);
    }
  }
  return FEHMM_OK;
}

int fehmm_bind_qps(fehmm_ctx* c, int n_qp, const int32_t* rve_of_qp) {
  if (!c || n_qp <= 0 || !rve_of_qp) return FEHMM_ERR_ARG;
  if (c->rve_n.empty()) return FEHMM_ERR_STATE;
  const int n_rve = (int)c->rve_n.size(), d = c->opt.dim;
  for (int q = 0; q < n_qp; ++q)
    if (rve_of_qp[q] < 0 || rve_of_qp[q] >= n_rve) return FEHMM_ERR_ARG;
  int rc;
  if ((rc = dupload(c->d_rve_n, c->rve_n.data(), c->rve_n.size())) ||
      (rc = dupload(c->d_rve_phase_off, c->rve_phase_off.data(), c->rve_phase_off.size())) ||
      (rc = dupload(c->d_phase, c->phase.data(), c->phase.size())) ||
      (rc = dupload(c->d_lame, c->lame.data(), c->lame.size())))
    return rc;
  std::vector<int64_t> off(n_qp);
  size_t total = 0;
  int nn_max = 0;
  std::vector<int> nodes(n_qp);
  for (int q = 0; q < n_qp; ++q) {
    const int n = c->rve_n[rve_of_qp[q]];
    int nn = 1;
    for (int k = 0; k < d; ++k) nn *= n;
    nodes[q] = nn;
    nn_max = std::max(nn_max, nn);
    off[q] = (int64_t)total;
    total += (size_t)nn * d;
  }
  // largest RVEs first so the persistent blocks finish together
  std::vector<int32_t> order(n_qp);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nodes[a] > nodes[b]; });
  if ((rc = dupload(c->d_qp_rve, rve_of_qp, (size_t)n_qp)) || (rc = dupload(c->d_order, order.data(), order.size())) ||
      (rc = dupload(c->d_w_off, off.data(), off.size())))
    return rc;
  dfree(c->d_w_cur);
  dfree(c->d_w_comm);
  if (cudaMalloc((void**)&c->d_w_cur, sizeof(double) * total) != cudaSuccess ||
      cudaMalloc((void**)&c->d_w_comm, sizeof(double) * total) != cudaSuccess) {
    cudaGetLastError();
    dfree(c->d_w_cur);
    dfree(c->d_w_comm);
    c->n_qp = 0;
    return FEHMM_ERR_OOM;
  }
  if (cudaMemset(c->d_w_cur, 0, sizeof(double) * total) != cudaSuccess ||
      cudaMemset(c->d_w_comm, 0, sizeof(double) * total) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  // kept tangent-transfer solutions: d*d fields of the point's dofs, in the solve's arithmetic type
  if (c->d_x_cur) cudaFree(c->d_x_cur);
  if (c->d_x_comm) cudaFree(c->d_x_comm);
  c->d_x_cur = c->d_x_comm = nullptr;
  c->x_bytes = 0;
  if (c->opt.transfer_warm) {
    const size_t xb = total * (size_t)(d * d) * (c->opt.precision == FEHMM_PREC_MIXED ? sizeof(float) : sizeof(double));
    if (cudaMalloc(&c->d_x_cur, xb) != cudaSuccess || cudaMalloc(&c->d_x_comm, xb) != cudaSuccess) {
      cudaGetLastError();
      if (c->d_x_cur) cudaFree(c->d_x_cur);
      if (c->d_x_comm) cudaFree(c->d_x_comm);
      c->d_x_cur = c->d_x_comm = nullptr;
      c->n_qp = 0;
      return FEHMM_ERR_OOM;
    }
    if (cudaMemset(c->d_x_cur, 0, xb) != cudaSuccess || cudaMemset(c->d_x_comm, 0, xb) != cudaSuccess)
      return FEHMM_ERR_CUDA;
    c->x_bytes = xb;
  }
  const int blocks = std::min(n_qp, c->num_sms);
  const bool mixed = c->opt.precision == FEHMM_PREC_MIXED;
  const size_t sb = d == 2 ? rve2d_scratch_bytes(nn_max, mixed, blocks) : rve3d_scratch_bytes(nn_max, mixed, blocks);
  if (sb > c->scratch_bytes) {
    if (c->d_scratch) cudaFree(c->d_scratch);
    c->d_scratch = nullptr;
    c->scratch_bytes = 0;
    if (cudaMalloc(&c->d_scratch, sb) != cudaSuccess) {
      cudaGetLastError();
      c->d_scratch = nullptr;
      return FEHMM_ERR_OOM;
    }
    c->scratch_bytes = sb;
  }
  c->n_qp = n_qp;
  c->nn_max = nn_max;
  c->w_total = total;
  c->w_off_h = off;
  return FEHMM_OK;
}

static int rve_solve_impl(fehmm_ctx* c, const double* F, double* P, double* A, double* W, int32_t* status,
                          int32_t* iters, int flags, const int32_t* list, const int32_t* count, void* stream);

int fehmm_rve_solve(fehmm_ctx* c, const double* F, double* P, double* A, double* W, int32_t* status, int32_t* iters,
                    int flags, void* stream) {
  return rve_solve_impl(c, F, P, A, W, status, iters, flags, nullptr, nullptr, stream);
}

int fehmm_rve_solve_list(fehmm_ctx* c, const double* F, double* P, double* A, double* W, int32_t* status,
                         int32_t* iters, int flags, const int32_t* list, const int32_t* count, void* stream) {
  if (!list || !count) return FEHMM_ERR_ARG;
  return rve_solve_impl(c, F, P, A, W, status, iters, flags, list, count, stream);
}

static int rve_solve_impl(fehmm_ctx* c, const double* F, double* P, double* A, double* W, int32_t* status,
                          int32_t* iters, int flags, const int32_t* list, const int32_t* count, void* stream) {
  if (!c || !F || !P || !status) return FEHMM_ERR_ARG;
  if (!(flags & FEHMM_SOLVE_NO_TANGENT) && !A) return FEHMM_ERR_ARG;
  if ((flags & FEHMM_SOLVE_ENERGY) && !W) return FEHMM_ERR_ARG;
  if (c->n_qp <= 0) return FEHMM_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  Rve2dArgs a{};
  a.n_qp = c->n_qp;
  a.nn_max = c->nn_max;
  a.order = list ? list : c->d_order;
  a.n_dev = count;
  a.qp_rve = c->d_qp_rve;
  a.rve_n = c->d_rve_n;
  a.rve_phase_off = c->d_rve_phase_off;
  a.phase = c->d_phase;
  a.rve_lame = c->d_lame;
  a.qp_w_off = c->d_w_off;
  a.w_in = (flags & FEHMM_SOLVE_FROM_COMMITTED) ? c->d_w_comm : c->d_w_cur;
  a.w_out = c->d_w_cur;
  const bool warm = c->opt.transfer_warm && c->d_x_cur;
  a.X_in = warm ? ((flags & FEHMM_SOLVE_FROM_COMMITTED) ? c->d_x_comm : c->d_x_cur) : nullptr;
  a.X_out = c->d_x_cur;
  a.F = F;
  a.P = P;
  a.A = (flags & FEHMM_SOLVE_NO_TANGENT) ? nullptr : A;
  a.W = W;
  a.status = status;
  a.iters = iters;
  a.queue = c->d_queue;
  a.scratch = c->d_scratch;
  a.newton_rtol = c->opt.newton_rtol;
  a.newton_atol = c->opt.newton_atol;
  a.cg_rtol = c->opt.cg_rtol;
  a.cond_rtol = c->opt.cond_rtol;
  a.max_newton = c->opt.max_newton;
  a.max_cg = c->opt.max_cg;
  a.max_cond_cg = c->opt.max_cond_cg;
  a.retry_stages = c->opt.retry_stages;
  a.flags = flags;
  const bool mixed = c->opt.precision == FEHMM_PREC_MIXED;
  a.mg = c->opt.precond == FEHMM_PRECOND_MULTIGRID ? 1 : 0;
  a.bc = c->opt.bc;
  a.law = c->opt.law;
  a.mg_omega = (float)c->opt.mg_omega;
  a.mg_reuse = c->opt.mg_reuse;
  a.scratch_stride = c->opt.dim == 2 ? rve2d_scratch_stride(c->nn_max, mixed) : 0;
  if (cudaMemsetAsync(c->d_queue, 0, sizeof(int32_t), s) != cudaSuccess) return FEHMM_ERR_CUDA;
  const int blocks = std::min(c->n_qp, c->num_sms);
  const cudaError_t err = c->opt.dim == 2 ? rve2d_launch(a, mixed, blocks, s) : rve3d_launch(a, mixed, blocks, s);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  c->launches += 1;
  return FEHMM_OK;
}

int fehmm_commit(fehmm_ctx* c, void* stream) {
  if (!c) return FEHMM_ERR_ARG;
  if (c->n_qp <= 0) return FEHMM_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(c->d_w_comm, c->d_w_cur, sizeof(double) * c->w_total, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      (c->x_bytes && cudaMemcpyAsync(c->d_x_comm, c->d_x_cur, c->x_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  return FEHMM_OK;
}

int fehmm_rollback(fehmm_ctx* c, void* stream) {
  if (!c) return FEHMM_ERR_ARG;
  if (c->n_qp <= 0) return FEHMM_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(c->d_w_cur, c->d_w_comm, sizeof(double) * c->w_total, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess ||
      (c->x_bytes && cudaMemcpyAsync(c->d_x_cur, c->d_x_comm, c->x_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  return FEHMM_OK;
}

int fehmm_transfer_state_all(fehmm_ctx* c, int which, void** dev_ptr, long long* n_bytes) {
  if (!c || !dev_ptr || (which != 0 && which != 1) || c->n_qp <= 0) return FEHMM_ERR_ARG;
  *dev_ptr = which ? c->d_x_comm : c->d_x_cur;
  if (n_bytes) *n_bytes = (long long)c->x_bytes;
  return FEHMM_OK;
}

int fehmm_fluctuation(fehmm_ctx* c, int q, int which, double** dev_ptr, int* n_values) {
  if (!c || !dev_ptr || q < 0 || q >= c->n_qp || (which != 0 && which != 1)) return FEHMM_ERR_ARG;
  *dev_ptr = (which ? c->d_w_comm : c->d_w_cur) + c->w_off_h[q];
  if (n_values) {
    const size_t end = (q + 1 < c->n_qp) ? (size_t)c->w_off_h[q + 1] : c->w_total;
    *n_values = (int)(end - (size_t)c->w_off_h[q]);
  }
  return FEHMM_OK;
}

int fehmm_fluctuation_all(fehmm_ctx* c, int which, double** dev_ptr, long long* n_values) {
  if (!c || !dev_ptr || (which != 0 && which != 1) || c->n_qp <= 0) return FEHMM_ERR_ARG;
  *dev_ptr = which ? c->d_w_comm : c->d_w_cur;
  if (n_values) *n_values = (long long)c->w_total;
  return FEHMM_OK;
}

int fehmm_macro_create(fehmm_ctx* c, const int32_t* n_el) {
  if (!c || !n_el) return FEHMM_ERR_ARG;
  const int d = c->opt.dim;
  for (int k = 0; k < d; ++k)
    if (n_el[k] < 1 || n_el[k] > 4096) return FEHMM_ERR_ARG;
  MacroArgs m{};
  m.dim = d;
  int nx[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) {
    nx[k] = n_el[k];
    m.nel[k] = n_el[k];
    m.h[k] = 1.0 / n_el[k];
  }
  m.nen = 1 << d;
  m.nq = 1 << d;
  m.n_el = nx[0] * nx[1] * nx[2];
  const int N0 = nx[0] + 1, N1 = nx[1] + 1, N2 = d == 3 ? nx[2] + 1 : 1;
  m.n_nodes = N0 * N1 * N2;
  m.n_qp = m.n_el * m.nq;
  // node-neighbour CSR (3^d stencil clipped at the boundary), d x d blocks
  const int nn = m.n_nodes;
  std::vector<std::vector<int>> nbr(nn);
  for (int k = 0; k < N2; ++k)
    for (int j = 0; j < N1; ++j)
      for (int i = 0; i < N0; ++i) {
        const int I = i + N0 * (j + N1 * k);
        for (int dk = (d == 3 ? -1 : 0); dk <= (d == 3 ? 1 : 0); ++dk)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              const int ii = i + di, jj = j + dj, kk = k + dk;
              if (ii < 0 || jj < 0 || kk < 0 || ii >= N0 || jj >= N1 || kk >= N2) continue;
              nbr[I].push_back(ii + N0 * (jj + N1 * kk));
            }
        std::sort(nbr[I].begin(), nbr[I].end());
      }
  std::vector<int32_t> rowptr((size_t)nn * d + 1, 0), col;
  std::vector<int32_t> node_base(nn);
  size_t pos = 0;
  for (int I = 0; I < nn; ++I) {
    node_base[I] = (int32_t)pos;
    for (int i = 0; i < d; ++i) {
      rowptr[(size_t)I * d + i] = (int32_t)pos;
      for (int J : nbr[I])
        for (int k = 0; k < d; ++k) col.push_back(J * d + k);
      pos += nbr[I].size() * d;
    }
  }
  rowptr[(size_t)nn * d] = (int32_t)pos;
  if (pos > (size_t)INT32_MAX) return FEHMM_ERR_UNSUPPORTED;
  const int nen = m.nen;
  std::vector<int32_t> blk_base((size_t)m.n_el * nen * nen), blk_stride((size_t)m.n_el * nen);
  auto corner = [&](int e, int a) {
    const int ex = e % nx[0], ey = (e / nx[0]) % nx[1], ez = e / (nx[0] * nx[1]);
    const int ox = ((a & 3) == 1 || (a & 3) == 2), oy = (a & 3) >= 2, oz = a >= 4;
    return (ex + ox) + N0 * ((ey + oy) + N1 * (ez + oz));
  };
  for (int e = 0; e < m.n_el; ++e)
    for (int I = 0; I < nen; ++I) {
      const int nI = corner(e, I);
      blk_stride[(size_t)e * nen + I] = (int32_t)(nbr[nI].size() * d);
      for (int J = 0; J < nen; ++J) {
        const int nJ = corner(e, J);
        const int rank = (int)(std::lower_bound(nbr[nI].begin(), nbr[nI].end(), nJ) - nbr[nI].begin());
        blk_base[((size_t)e * nen + I) * nen + J] = node_base[nI] + rank * d;
      }
    }
  int rc;
  if ((rc = dupload(c->d_rowptr, rowptr.data(), rowptr.size())) || (rc = dupload(c->d_col, col.data(), col.size())) ||
      (rc = dupload(c->d_blk_base, blk_base.data(), blk_base.size())) ||
      (rc = dupload(c->d_blk_stride, blk_stride.data(), blk_stride.size())))
    return rc;
  m.blk_base = c->d_blk_base;
  m.blk_stride = c->d_blk_stride;
  std::vector<uint8_t> nofix((size_t)nn * d, 0);
  if ((rc = dupload(c->d_fixed, nofix.data(), nofix.size()))) return rc;
  dfree(c->d_solve_work);
  const size_t wd = macro_solve_work_doubles(nn * d, c->num_sms);
  if (cudaMalloc((void**)&c->d_solve_work, sizeof(double) * wd) != cudaSuccess) {
    cudaGetLastError();
    c->d_solve_work = nullptr;
    return FEHMM_ERR_OOM;
  }
  c->macro = m;
  c->macro_rows = nn * d;
  c->macro_nnz = (int)pos;
  c->has_macro = true;
  return FEHMM_OK;
}

int fehmm_macro_qp_F(fehmm_ctx* c, const double* u, double* F, void* stream) {
  if (!c || !u || !F) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  MacroArgs m = c->macro;
  m.u = u;
  m.F = F;
  if (macro_qp_F_launch(m, (cudaStream_t)stream) != cudaSuccess) return FEHMM_ERR_CUDA;
  c->launches += 1;
  return FEHMM_OK;
}

int fehmm_macro_assemble(fehmm_ctx* c, const double* P, const double* A, double* f, double* K_vals, void* stream) {
  if (!c || !P || !f || (A && !K_vals)) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  MacroArgs m = c->macro;
  m.P = P;
  m.A = A;
  m.f = f;
  m.K = K_vals;
  if (cudaMemsetAsync(f, 0, sizeof(double) * (size_t)m.n_nodes * m.dim, s) != cudaSuccess) return FEHMM_ERR_CUDA;
  if (A && cudaMemsetAsync(K_vals, 0, sizeof(double) * (size_t)c->macro_nnz, s) != cudaSuccess) return FEHMM_ERR_CUDA;
  int launches = 0;
  const cudaError_t err = macro_assemble_launch(m, s, &launches);
  c->launches += launches;
  return err == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

int fehmm_macro_set_dirichlet(fehmm_ctx* c, int n_fixed, const int32_t* dofs, const double* values) {
  if (!c || n_fixed < 0 || (n_fixed > 0 && (!dofs || !values))) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  std::vector<uint8_t> mask((size_t)c->macro_rows, 0);
  std::vector<double> full((size_t)c->macro_rows, 0.0);
  for (int k = 0; k < n_fixed; ++k) {
    if (dofs[k] < 0 || dofs[k] >= c->macro_rows) return FEHMM_ERR_ARG;
    mask[dofs[k]] = 1;
    full[dofs[k]] = values[k];
  }
  int rc;
  if ((rc = dupload(c->d_fixed, mask.data(), mask.size())) || (rc = dupload(c->d_fixed_dofs, dofs, (size_t)n_fixed)) ||
      (rc = dupload(c->d_fixed_vals, values, (size_t)n_fixed)) || (rc = dupload(c->d_dir_full, full.data(), full.size())))
    return rc;
  c->n_fixed = n_fixed;
  return FEHMM_OK;
}

int fehmm_macro_apply_dirichlet(fehmm_ctx* c, double* u, double* du, double scale, void* stream) {
  if (!c || !u) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  if (macro_dirichlet_launch(u, du, c->macro_rows, c->d_fixed_dofs, c->d_fixed_vals, c->n_fixed, scale,
                             (cudaStream_t)stream) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  c->launches += 1;
  return FEHMM_OK;
}

int fehmm_macro_dirichlet_load(fehmm_ctx* c, const double* K_vals, double dscale, double* g, void* stream) {
  if (!c || !K_vals || !g) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  if (!c->d_dir_full) {  // no Dirichlet data: the load is zero
    if (cudaMemsetAsync(g, 0, sizeof(double) * (size_t)c->macro_rows, (cudaStream_t)stream) != cudaSuccess) {
      cudaGetLastError();
      return FEHMM_ERR_CUDA;
    }
    return FEHMM_OK;
  }
  if (macro_spmv_launch(c->d_rowptr, c->d_col, K_vals, c->d_dir_full, dscale, g, c->macro_rows,
                        (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  c->launches += 1;
  return FEHMM_OK;
}

int fehmm_macro_update(fehmm_ctx* c, double* u, const double* du, void* stream) {
  if (!c || !u || !du) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  if (macro_update_launch(u, du, c->macro_rows, (cudaStream_t)stream) != cudaSuccess) return FEHMM_ERR_CUDA;
  c->launches += 1;
  return FEHMM_OK;
}

int fehmm_macro_solve(fehmm_ctx* c, const double* K_vals, const double* f, double* du, double* info, double rtol,
                      int max_it, void* stream) {
  if (!c || !K_vals || !f || !du || !info || !(rtol > 0) || max_it <= 0) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  MacroSolveArgs a{};
  a.n = c->macro_rows;
  a.rowptr = c->d_rowptr;
  a.col = c->d_col;
  a.K = K_vals;
  a.f = f;
  a.fixed = c->d_fixed;
  a.du = du;
  a.work = c->d_solve_work;
  a.out = info;
  a.rtol = rtol;
  a.max_it = max_it;
  if (macro_solve_launch(a, macro_solve_blocks(c->num_sms, c->macro_rows), (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_CUDA;
  }
  c->launches += 1;
  return FEHMM_OK;
}

int fehmm_macro_csr(fehmm_ctx* c, const int32_t** rowptr, const int32_t** col, int* n_rows, int* nnz) {
  if (!c) return FEHMM_ERR_ARG;
  if (!c->has_macro) return FEHMM_ERR_STATE;
  if (rowptr) *rowptr = c->d_rowptr;
  if (col) *col = c->d_col;
  if (n_rows) *n_rows = c->macro_rows;
  if (nnz) *nnz = c->macro_nnz;
  return FEHMM_OK;
}

long long fehmm_launch_count(const fehmm_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"

// ------------------------------------------------------------------------------ autotuner
namespace {

// Cache key: everything the choice depends on besides the deformation (problem class, grids,
// device).  One text line per tuned configuration: "<key>\t<precond> <mg_omega> <cg_rtol>
// <mg_reuse> <seconds per RVE solve>"; the last matching line wins.
std::string tune_key(const fehmm_ctx* c) {
  std::vector<int> grids(c->rve_n.begin(), c->rve_n.end());
  std::sort(grids.begin(), grids.end());
  grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
  cudaDeviceProp prop;
  const char* dev = cudaGetDeviceProperties(&prop, c->device) == cudaSuccess ? prop.name : "unknown";
  char buf[256];
  snprintf(buf, sizeof(buf), "dim=%d prec=%d law=%d bc=%d grids=", c->opt.dim, c->opt.precision, c->opt.law, c->opt.bc);
  std::string key(buf);
  for (size_t k = 0; k < grids.size(); ++k) key += (k ? "," : "") + std::to_string(grids[k]);
  key += " dev=";
  key += dev;
  for (char& ch : key)
    if (ch == '\t' || ch == '\n') ch = ' ';
  return key;
}

bool tune_cache_lookup(const char* path, const std::string& key, fehmm_tune_result* r) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  bool found = false;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    if (key != line) continue;
    fehmm_tune_result t{};
    if (sscanf(tab + 1, "%d %lf %lf %d %lf", &t.precond, &t.mg_omega, &t.cg_rtol, &t.mg_reuse, &t.seconds_per_solve) ==
        5) {
      *r = t;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_store(const char* path, const std::string& key, const fehmm_tune_result& r) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d %.17g %.17g %d %.9g\n", key.c_str(), r.precond, r.mg_omega, r.cg_rtol, r.mg_reuse,
          r.seconds_per_solve);
  fclose(f);
}

}  // namespace

extern "C" {

int fehmm_autotune(fehmm_ctx* c, const double* F, int n_sample, const char* cache_path, fehmm_tune_result* out,
                   void* stream) {
  if (!c || !F) return FEHMM_ERR_ARG;
  if (c->n_qp <= 0) return FEHMM_ERR_STATE;
  const std::string key = tune_key(c);
  fehmm_tune_result best{};
  if (tune_cache_lookup(cache_path, key, &best)) {
    fehmm_options o = c->opt;
    o.precond = best.precond;
    o.mg_omega = best.mg_omega;
    o.cg_rtol = best.cg_rtol;
    o.mg_reuse = best.mg_reuse;
    if (!valid_options(&o)) return FEHMM_ERR_ARG;
    c->opt = o;
    best.from_cache = 1;
    best.candidates = 0;
    if (out) *out = best;
    return FEHMM_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int d = c->opt.dim, n_qp = c->n_qp;
  const int ns = n_sample > 0 ? std::min(n_sample, n_qp) : std::min(n_qp, 2 * c->num_sms);
  // an evenly strided sample of the bound points (covers every grid size of a mixed batch)
  std::vector<int32_t> list(ns);
  for (int k = 0; k < ns; ++k) list[k] = (int32_t)(((long long)k * n_qp) / ns);
  int32_t* d_list = nullptr;
  int32_t* d_status = nullptr;
  double *d_P = nullptr, *d_A = nullptr, *d_save = nullptr;
  void* d_xsave = nullptr;
  int32_t cnt = ns;
  int rc = FEHMM_OK;
  const size_t nA = (size_t)n_qp * d * d * d * d;
  if (cudaMalloc((void**)&d_list, sizeof(int32_t) * (ns + 1)) != cudaSuccess ||
      cudaMalloc((void**)&d_status, sizeof(int32_t) * n_qp) != cudaSuccess ||
      cudaMalloc((void**)&d_P, sizeof(double) * (size_t)n_qp * d * d) != cudaSuccess ||
      cudaMalloc((void**)&d_A, sizeof(double) * nA) != cudaSuccess ||
      cudaMalloc((void**)&d_save, sizeof(double) * c->w_total) != cudaSuccess ||
      (c->x_bytes && cudaMalloc(&d_xsave, c->x_bytes) != cudaSuccess)) {
    cudaGetLastError();
    rc = FEHMM_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == FEHMM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = FEHMM_ERR_CUDA;
  if (rc == FEHMM_OK &&
      (cudaMemcpyAsync(d_list, list.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(d_list + ns, &cnt, sizeof(int32_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(d_save, c->d_w_cur, sizeof(double) * c->w_total, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
       (c->x_bytes && cudaMemcpyAsync(d_xsave, c->d_x_cur, c->x_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) ||
       cudaStreamSynchronize(s) != cudaSuccess))
    rc = FEHMM_ERR_CUDA;
  // candidates: the preconditioner, the smoother damping (below the positive-definiteness bound of
  // each element type), the coarse-level reuse (3D), the Newton-correction PCG tolerance
  struct Cand {
    int precond;
    double omega, cg_rtol;
    int reuse;
  };
  std::vector<Cand> cands;
  const fehmm_options base = c->opt;
  const double cgr[3] = {base.cg_rtol, base.cg_rtol * 10.0, base.cg_rtol * 0.1};
  const double om2[4] = {0.5, 0.6, 0.7, 0.8}, om3[4] = {0.45, 0.55, 0.6, 0.65};
  for (int kc = 0; kc < 3; ++kc) {
    if (!(cgr[kc] > 0 && cgr[kc] < 0.5)) continue;
    for (int ko = 0; ko < 4; ++ko)
      for (int reuse = (d == 3 ? 0 : 1); reuse <= 1; ++reuse)
        cands.push_back({FEHMM_PRECOND_MULTIGRID, d == 2 ? om2[ko] : om3[ko], cgr[kc], reuse});
    cands.push_back({FEHMM_PRECOND_BLOCK_JACOBI, base.mg_omega, cgr[kc], base.mg_reuse});
  }
  double best_t = 1e300;
  int n_ok = 0;
  std::vector<int32_t> st(n_qp);
  for (size_t k = 0; rc == FEHMM_OK && k < cands.size(); ++k) {
    fehmm_options o = base;
    o.precond = cands[k].precond;
    o.mg_omega = cands[k].omega;
    o.cg_rtol = cands[k].cg_rtol;
    o.mg_reuse = cands[k].reuse;
    if (!valid_options(&o)) continue;
    c->opt = o;
    float ms = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {  // the first run warms up, the second is timed
      if (cudaMemsetAsync(d_status, 0xff, sizeof(int32_t) * n_qp, s) != cudaSuccess ||
          cudaEventRecord(e0, s) != cudaSuccess) {
        rc = FEHMM_ERR_CUDA;
        break;
      }
      const int r = rve_solve_impl(c, F, d_P, d_A, nullptr, d_status, nullptr, FEHMM_SOLVE_FROM_COMMITTED, d_list,
                                   d_list + ns, stream);
      if (r != FEHMM_OK || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        rc = r != FEHMM_OK ? r : FEHMM_ERR_CUDA;
        break;
      }
      cudaEventElapsedTime(&ms, e0, e1);
      if (cudaMemcpy(st.data(), d_status, sizeof(int32_t) * n_qp, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = FEHMM_ERR_CUDA;
        break;
      }
      for (int q : list) ok = ok && st[q] == FEHMM_RVE_OK;
    }
    if (rc != FEHMM_OK) break;
    if (!ok) continue;  // a setting that does not converge on the sample is never chosen
    ++n_ok;
    const double t = ms * 1e-3 / ns;
    if (t < best_t) {
      best_t = t;
      best.precond = o.precond;
      best.mg_omega = o.mg_omega;
      best.cg_rtol = o.cg_rtol;
      best.mg_reuse = o.mg_reuse;
      best.seconds_per_solve = t;
    }
  }
  // the current fluctuations (and kept transfer solutions) as before the trials
  if (rc == FEHMM_OK &&
      (cudaMemcpyAsync(c->d_w_cur, d_save, sizeof(double) * c->w_total, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
       (c->x_bytes && cudaMemcpyAsync(c->d_x_cur, d_xsave, c->x_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)))
    rc = FEHMM_ERR_CUDA;
  if (rc == FEHMM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = FEHMM_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(d_list);
  dfree(d_status);
  dfree(d_P);
  dfree(d_A);
  dfree(d_save);
  if (d_xsave) cudaFree(d_xsave);
  if (rc == FEHMM_OK && n_ok == 0) rc = FEHMM_ERR_UNSUPPORTED;  // nothing converged: keep the options
  if (rc != FEHMM_OK) {
    cudaGetLastError();
    c->opt = base;
    return rc;
  }
  fehmm_options o = base;
  o.precond = best.precond;
  o.mg_omega = best.mg_omega;
  o.cg_rtol = best.cg_rtol;
  o.mg_reuse = best.mg_reuse;
  c->opt = o;
  best.from_cache = 0;
  best.candidates = (int)cands.size();
  tune_cache_store(cache_path, key, best);
  if (out) *out = best;
  return FEHMM_OK;
}

const char* fehmm_status_str(int code) {
  switch (code) {
    case FEHMM_OK: return "ok";
    case FEHMM_ERR_ARG: return "invalid argument";
    case FEHMM_ERR_CUDA: return "CUDA error";
    case FEHMM_ERR_OOM: return "out of device memory";
    case FEHMM_ERR_STATE: return "call out of order";
    case FEHMM_ERR_UNSUPPORTED: return "unsupported configuration";
    case FEHMM_ERR_TOO_LARGE: return "size exceeds the static scratch of the no-allocation entry point";
    default: return code > 0 ? "some RVE solves did not converge" : "unknown status";
  }
}

}  // extern "C"
