// Launch arguments of the batched RVE kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fehmm {

struct Rve2dArgs {
  int n_qp;                     // quadrature points in the batch
  int nn_max;                   // largest n^2 over the batch (sizes shared memory)
  const int32_t* order;         // [n_qp] processing order (largest RVE first)
  const int32_t* qp_rve;        // [n_qp] microstructure of each point
  const int32_t* rve_n;         // [n_rve] grid size
  const int64_t* rve_phase_off; // [n_rve] offset of the phase map
  const uint8_t* phase;         // concatenated phase maps
  const double* rve_lame;       // [n_rve][kMaxPhase][2] (lambda, mu)
  const int64_t* qp_w_off;      // [n_qp] offset (doubles) of each fluctuation field
  const double* w_in;           // start fluctuations
  double* w_out;                // result fluctuations (may alias w_in)
  const double* F;             // [n_qp][4]
  double* P;                    // [n_qp][4]
  double* A;                    // [n_qp][16] or null
  double* W;                    // [n_qp] or null
  int32_t* status;              // [n_qp]
  int32_t* iters;               // [n_qp][4] or null
  int32_t* queue;               // work counter, zero at launch
  void* scratch;                // per-block global scratch (FP64 mode)
  double newton_rtol, newton_atol, cg_rtol, cond_rtol;
  int max_newton, max_cg, max_cond_cg, flags;
  int retry_stages;      // > 1: load continuation from w = 0 after a failed Newton solve
  int mg;                // 1: multigrid-preconditioned PCG where the grid allows it (2D)
  long long scratch_stride;  // per-block scratch, in elements of the kernel's arithmetic type (2D)
  const int32_t* n_dev;  // optional: number of work items in device memory (order = a qp list)
  int fixed_n;        // fixed-layout launches only: grid size of every RVE
  int phase_per_qp;   // fixed-layout launches only: 1 = one phase map per qp, 0 = one shared
  int bc;             // 0 periodic (node 0 pinned), 1 KUBC (nodes on the planes x_c = 0 pinned)
  int law;            // 0 neo-Hookean, 1 St. Venant-Kirchhoff
  float mg_omega;     // smoother damping of the multigrid V-cycle
  int mg_reuse;       // 3D: reuse the coarse levels over the Newton iterations of a solve
  const void* X_in;   // kept tangent-transfer solutions (TA) to start from, or null (start from 0);
                      // per point at (2D: 4, 3D: 9) x qp_w_off[qp], layout [d*d][NN][d]
  void* X_out;        // where the new transfer solutions go (may alias X_in; null: not kept)
};

size_t rve2d_smem_bytes(int nn_max, bool mixed);
size_t rve2d_scratch_bytes(int nn_max, bool mixed, int n_blocks);
long long rve2d_scratch_stride(int nn_max, bool mixed);
int rve2d_threads();
cudaError_t rve2d_launch(const Rve2dArgs& a, bool mixed, int n_blocks, cudaStream_t stream);
cudaError_t rve2d_launch_fixed_fp64(const Rve2dArgs& a, int n_blocks, cudaStream_t stream);
size_t rve3d_smem_bytes(int nn_max, bool mixed);
size_t rve3d_scratch_bytes(int nn_max, bool mixed, int n_blocks);
cudaError_t rve3d_launch(const Rve2dArgs& a, bool mixed, int n_blocks, cudaStream_t stream);

struct MacroArgs {
  int dim;
  int nel[3];           // elements per axis
  int n_el, n_nodes, n_qp, nq, nen;
  double h[3];
  const double* u;      // [n_nodes*dim]
  double* F;            // [n_qp][d*d]
  const double* P;      // [n_qp][d*d]
  const double* A;      // [n_qp][d^4]
  double* f;            // [n_nodes*dim]
  double* K;            // [nnz]
  const int32_t* blk_base;    // [n_el][nen][nen] CSR position of the (I,J) block's (0,0) entry
  const int32_t* blk_stride;  // [n_el][nen] row stride (entries) between the dim rows of node I
};

struct MacroSolveArgs {
  int n;                    // rows (macro dofs)
  const int32_t* rowptr;    // CSR pattern
  const int32_t* col;
  const double* K;          // CSR values
  const double* f;          // macro residual
  const uint8_t* fixed;     // [n] 1 = Dirichlet dof
  double* du;               // [n] correction (output)
  double* work;             // 6n + 4*blocks doubles (two alternating partial-sum buffers)
  double* out;              // [3]: |f_free|_2, iterations, status (0 ok, 1 cap, 2 breakdown)
  double rtol;
  int max_it;
};

size_t macro_solve_work_doubles(int n, int blocks);
int macro_solve_blocks(int num_sms, long long n_rows);
cudaError_t macro_solve_launch(const MacroSolveArgs& a, int blocks, cudaStream_t stream);

cudaError_t macro_qp_F_launch(const MacroArgs& m, cudaStream_t stream);
cudaError_t macro_dirichlet_launch(double* u, double* du, int n, const int32_t* dofs, const double* vals, int n_fixed,
                                   double scale, cudaStream_t stream);
cudaError_t macro_update_launch(double* u, const double* du, int n, cudaStream_t stream);
cudaError_t macro_spmv_launch(const int32_t* rowptr, const int32_t* col, const double* K, const double* x,
                              double scale, double* y, int n, cudaStream_t stream);
cudaError_t macro_assemble_launch(const MacroArgs& m, cudaStream_t stream, int* launches);

}  // namespace fehmm
