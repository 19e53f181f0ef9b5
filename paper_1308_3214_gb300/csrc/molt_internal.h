// molt_internal.h -- launchers shared by the C-ABI layer and the kernel unit.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>
#include "molt.h"
#include "molt_kernels.cuh"

namespace molt {

constexpr int kMaxP = 5;            // highest order parameter P (order 2P)
constexpr int64_t kMaxLine = 12288;  // longest line of the single-problem sweeps (two float64
                                     // line buffers of one line fill most of shared memory)

// Host constants of the scheme (molt_host.cu).
double term_weight(int p, int m, double beta);     // weight of C^m D^{p-m} in the update
double beta_max_of(int P);                         // Table 1; -1 outside 1..5
// F = sum f_ijk D_x^i D_y^j D_z^k, degree <= P per axis, index i + (P+1)(j + (P+1)k)
bool expand_coefficients(int ndim, int P, double beta, std::vector<double> &out);
double quad_R(double nu);                          // second-difference weight of the quadratic rule
void axis_constants(double nu, int64_t n, int bc, int quad, AxisDev &A);

// Message for mol_last_error(NULL) (molt_api.cu).
void set_global_error(const std::string &msg);

// tbytes: 4 -> float32 sweeps (pair levels), 8 -> float64 throughout.
cudaError_t launch_powers(int tbytes, int bc, bool contig, const AxisDev &A, const PassGeom &G,
                          const PowersParams &p, cudaStream_t s);
cudaError_t launch_horner(int tbytes, int bc, bool contig, const AxisDev &A, const PassGeom &G,
                          const HornerParams &p, cudaStream_t s);
cudaError_t launch_to_pair(const double *x, float *hi, float *lo, int64_t N, cudaStream_t s);
cudaError_t launch_from_pair(const float *hi, const float *lo, double *x, int64_t N, cudaStream_t s);
// two levels in one launch where every field is 16-byte aligned, else two
cudaError_t launch_to_pair2(const double *x0, float *hi0, float *lo0, const double *x1, float *hi1, float *lo1,
                            int64_t N, cudaStream_t s);
cudaError_t launch_from_pair2(const float *hi0, const float *lo0, double *x0, const float *hi1, const float *lo1,
                              double *x1, int64_t N, cudaStream_t s);
cudaError_t launch_from_f32(const float *f, double *x, int64_t N, cudaStream_t s);

// Test hooks (molt_host.cu; set through mol_debug_fail_alloc /
// mol_debug_allow_unstable): true when the next device allocation is to fail
// as if the device were full; true when beta above beta_max is accepted.
bool alloc_injected_failure();
bool unstable_allowed();

// Checkpoint-and-recompute history gradient (molt_host.cu), shared by the
// single-problem and batch handles through their own field operations.
struct HistoryOps {
    void *ctx;
    int64_t N;                                                  // doubles per field
    mol_status (*start)(void *, const double *u0, double *u1, cudaStream_t);
    mol_status (*step)(void *, double *prev, double *cur, int64_t nsteps, cudaStream_t);
    // m steps from (prev, cur), unchanged; the new levels into states[0..m)
    mol_status (*step_emit)(void *, const double *prev, const double *cur, int64_t m, double *states, cudaStream_t);
    // un = ea u + eb up + ec F^T u (+ add)
    mol_status (*update_T)(void *, const double *u, const double *up, double *un, double ea, double eb, double ec,
                           const double *add, cudaStream_t);
    mol_status (*fail)(void *, mol_status, const char *);
};
mol_status history_gradient_run(const HistoryOps &o, const double *u0, int64_t nsteps, int64_t K, mol_grad_fn fn,
                                void *user, double *grad, cudaStream_t s);

// Allow every pass kernel the largest dynamic shared-memory carve-out.
cudaError_t configure_kernels();

// Bytes of dynamic shared memory a pass needs.
size_t pass_smem_bytes(bool horner, int tbytes, int W, int ls, int n, int dps = 1);

// Line stride in shared memory for W lines of segment stride ms.
int line_stride(int ms, int W, int tbytes);

// Register-resident kernels (molt_regs.cu).  The *_plan functions say whether
// a line of n points is supported and with which segment decomposition.
bool regs_contig_plan(int tbytes, int bc, int n, int *rpt);
// pref_rpt: 0 = default segment length (or 32 for float lines, a tuner
// choice); max_warps: segments per CTA at most (1..8)
bool regs_strided_plan(int tbytes, int bc, int n, int *rpt, int *S, int *K, int pref_rpt = 0, int max_warps = 8);
size_t regs_strided_smem(int tbytes, int S, int rpt, bool horner);
cudaError_t launch_contig(int tbytes, int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p,
                          cudaStream_t s);
cudaError_t launch_strided(int tbytes, int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p,
                           cudaStream_t s);
cudaError_t configure_regs_kernels();
// The strided powers pass with one neighbour exchange per sweep (float32):
// true when a line of n points with segments of rpt points and decay d is
// computed by it exactly to well below float32 rounding (molt_strided_nb.cuh).
bool regs_strided_nb_plan(double d, int n, int rpt);
// The row-split x pass with one neighbour exchange per sweep: W = 2 warps per
// row with one hop (dropped inflows d^(RPT-1) <= 2^-27, below 1/8 of a float32
// ulp) or W = 4 with two hops (d^(2 RPT - 1) <= 2^-27).
bool rows_nb_plan(double d, int n, int rpt, int W);
// stage: 0 direct loads and stores, 1 the pair level's tile through TMA into
// shared memory, 2 each output power staged in shared memory and written by
// TMA tensor stores, 3 both
cudaError_t launch_strided_nb(int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s,
                              int stage = 0);
// The strided Horner pass (several outputs, float32) with one neighbour
// exchange per sweep, under the same condition on d; gtile: the g fields'
// rows staged in shared memory once per CTA (where two CTAs per SM still fit).
cudaError_t launch_strided_nb_h(int bc, int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p,
                                cudaStream_t s, bool gtile);
// The transposed strided powers (the adjoint step's y pass, Dirichlet,
// float32) with one neighbour exchange per sweep, under the same condition.
cudaError_t launch_strided_nb_T(int rpt, const AxisDev &A, const LineSet &L, const ProgParams &p, cudaStream_t s);
// 1 if a bounded wait of a register kernel gave up since the last call (and
// clears it), 0 if not, -1 if the flag could not be read; synchronizes s.
int regs_timeout_take(cudaStream_t s);
// A kernel whose bounded wait cannot succeed (mol_wait_selftest).
cudaError_t launch_wait_selftest(long long limit_cycles, cudaStream_t s);
bool regs_res_plan(int tbytes, int n, int ng, int *rpt);
bool regs_rows_plan(int tbytes, int n, int ng, int W, int *rpt);
cudaError_t launch_rows(int bc, int rpt, int ng, int W, const AxisDev &A, const LineSet &L, const ProgParams &p,
                        cudaStream_t s);
cudaError_t launch_res(int bc, int rpt, int ng, int warps, const AxisDev &A, const LineSet &L, const ProgParams &p,
                       cudaStream_t s);

}  // namespace molt
