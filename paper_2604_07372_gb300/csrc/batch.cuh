// Instance table of the batched and served forms (shared by batch.cu and server.cu).
#pragma once

#include "common.cuh"

namespace nsrgs {

// One instance as the batched kernels see it (device memory, written by the host).
// Phase of a batched / served instance after its spectral passes: the blocks of
// its basis are turned into X^0 (extends the PHASE_* values of the control block).
constexpr int PHASE_POLAR = 5;
// First, orthonormalising spectral pass (W = V^0, no A-stream), after admission.
constexpr int PHASE_SPEC0 = 6;
// Orthonormalising pass of a restart: the spectral passes converged to a basis
// that failed the algebraic top-d test and start again from V^0 under a larger
// shift (spec_shift_after); like PHASE_SPEC0, but V^0 is regenerated, not read.
constexpr int PHASE_SPECR = 7;

// Per-instance float64 scratch of the spectral passes (doubles, D <= 4).
constexpr int kScrWW = 0;     // W^T W accumulator, D x D
constexpr int kScrVW = 16;    // V^T W accumulator, D x D
constexpr int kScrRinv = 32;  // R^{-1} of the Cholesky of W^T W
constexpr int kScrH = 48;     // H = V^T W
constexpr int kScrH2 = 64;    // ||H||_F^2
constexpr int kScrRes = 65;   // residual accumulator
constexpr int kScrShift = 66; // shift c of W = A_off V + c V
constexpr int kScrBytes = 1024;

struct BatchDesc {
  const uint8_t* packed;  // packed A (panel layout)
  float* X[2];            // ping-pong iterates / spectral bases, padded to n*d + 64 rows
  float* Y;               // A-stream accumulator, padded
  float* W;               // spectral scratch, padded
  Ctl* ctl;               // control block: phase, counters, flags
  double* scr;            // spectral-pass scratch (kScr* offsets)
  float* Xout;            // caller's X: X^0 when start_given, the result when done
  PanelGeom g;
  float eta;
  int T;
  int K;
  int smax;               // spectral passes cap
  int start_given;        // 1: X^0 comes from Xout, no spectral initialisation
  int safeguard;          // 1: safeguarded Newton-Schulz start (beyond the paper)
  int sparse;             // 1: block-sparse rows (streamed by the row kernel, no panel steps)
  int resident;           // persistent form: the panels fit a CTA's stage space (kept in shared memory)
  double tol;             // stop when the update norm falls below it (0: run T iterations)
  double spec_tol;        // spectral residual target
};

struct BatchReport {
  int phase;
  int spec_iters;
  int iters;
  unsigned int flags;
  double last_upd;
  double spec_res;
};

size_t batch_instance_bytes(int n, int d);
size_t batch_table_bytes(int count);
void fill_instance(BatchDesc& ds, uint8_t* region, int n, int d);
// The row kernel over the block-sparse instances: rbase[i] = first global row of
// instance i (instances without block-sparse storage add no rows).
cudaError_t batch_bcsr_stream(const BatchDesc* descs, const long long* rbase, int count, int d, int elem_bf16,
                              long long total_rows, cudaStream_t st);
cudaError_t batch_stream(const BatchDesc* descs, const long long* base, int count, int d, int storage,
                         cudaStream_t st, bool prepare);
cudaError_t batch_admit(const BatchDesc* descs, int count, int d, int* nspec, cudaStream_t st);
cudaError_t batch_spec(const BatchDesc* descs, const long long* bbase, int count, int d, long long total_blocks,
                       int* nspec, cudaStream_t st);
cudaError_t batch_block(const BatchDesc* descs, const long long* bbase, int count, int d, long long total_blocks,
                        cudaStream_t st);
cudaError_t batch_report(const BatchDesc* descs, int count, BatchReport* out, cudaStream_t st);
cudaError_t batch_reset(const BatchDesc* descs, int count, int* nspec, cudaStream_t st);
// Persistent form (batch_persist.cu): one launch, a CTA per instance at a time.
bool persist_fits_resident(const PanelGeom& g);
cudaError_t batch_persist(const BatchDesc* descs, const int* order, int count, int* next, int d, int storage,
                          cudaStream_t st, bool prepare);

}  // namespace nsrgs
