// pmp_launch.h -- host-side launchers of the PMP kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "pmp_device.cuh"

// Calls CALL with the compile-time constant RR = R_ (the stencil half-width).
#define PMP_DISPATCH_R(R_, CALL)                         \
    switch (R_) {                                        \
    case 1: { constexpr int RR = 1; CALL; } break;       \
    case 2: { constexpr int RR = 2; CALL; } break;       \
    case 3: { constexpr int RR = 3; CALL; } break;       \
    case 4: { constexpr int RR = 4; CALL; } break;       \
    case 5: { constexpr int RR = 5; CALL; } break;       \
    default: { constexpr int RR = 6; CALL; } break;      \
    }

namespace pmp {

// Device pointers into a pass's workspace (the plan and the per-cell arrays).
// Particle t of the processing order owns slots [t * cap, t * cap + counts[t]).
struct PlanPtrs {
    const unsigned *perm;             // processing order (null: index order)
    unsigned *counts;                 // [n + 1] kernel cells per processed particle
    unsigned long long *slots;        // [n * cap] packed cell + omega count
    unsigned long long *hosts;        // [n] packed host cell, by particle index
    float4 *fr;                       // [n] fractional position in the host cell (FP32)
    double *wts;                      // sink: [n][3][2R+1] per-axis Gaussian factors
    double *grec;                     // sink: [valid cells][4] G records
    double *gcs;                      // sink: [valid cells] rho c_s
    double *drec;                     // sink: [valid cells][4] D records
    double *dtr;                      // sink: [valid cells] rho - rho_Tr
    double *deta;                     // sink: [valid cells] eta (1 until Step 3 limits the cell)
    double *pa;                       // sink, fused ATOMIC deposit: [n * cap] each pair's removal a, by slot
    unsigned long long cap;           // slots per particle
};

void launch_prologue(const Box &S, const Parts &p, unsigned *keys, unsigned *ids, const PlanPtrs &pl, DevStatus *st,
                     cudaStream_t stream);
void launch_plan(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                 cudaStream_t stream);
void launch_gather(const KParams &P, const Box &S, const double *u, const Parts &p, const PlanPtrs &pl, double *G,
                   DevStatus *st, cudaStream_t stream);
// Supernova kind: plan and gather in one launch (same slots, counts and rows
// as launch_plan followed by launch_gather).
void launch_plan_gather_fb(const KParams &P, const Box &S, const double *u, const Parts &p, const PlanPtrs &pl,
                           double *G, DevStatus *st, cudaStream_t stream);
// Sink kind, ATOMIC mode: plan, gather and the scratch deposit (-a per pair
// into scr, zeroed) in one launch; the per-cell records must be written
// first, launch_sink_spread completes Step 1.
void launch_pass1_sink(const KParams &P, const Box &S, const double *u, const Box &B, double *scr, const Parts &p,
                       const PlanPtrs &pl, double *G, DevStatus *st, cudaStream_t stream);
// E (optional): App. A.1 error-bound buffer, the buffer's layout, zeroed.
// scr (optional, sinks): one-field scratch with the buffer's layout, zeroed;
// the deposit then sums only -a per cell into it and launch_sink_spread
// completes Step 1.
void launch_deposit_atomic(const KParams &P, const Box &S, const double *u, const Box &B, double *b, const Parts &p,
                           const double *G, const PlanPtrs &pl, double *E, double *scr, cudaStream_t stream);
// Sorted deposit, first part: every pair's deposition value (the same
// function and operations as the atomic deposit).  Pair q of the particle at
// processing position t (particle s = perm[t]) is stored at
// pv[(offsets[t] + q) * 5 + f], so that the values of nearby particles lie
// together; the pair sort's input lists are in particle-index order: its
// buffer cell at keys[koffsets[s] + q] and offsets[t] + q at vals[koffsets[s]
// + q].  offsets / koffsets: exclusive prefix sums of the pair counts in
// processing / index order.
void launch_pair_values(const KParams &P, const Box &S, const double *u, const Box &B, const Parts &p,
                        const double *G, const PlanPtrs &pl, const unsigned long long *offsets,
                        const unsigned long long *koffsets, double *pv, unsigned *keys, unsigned *vals,
                        cudaStream_t stream);
// counts_idx[perm[t]] = counts[t] for t < n, counts_idx[n] = 0 (the pair
// counts in particle-index order).
void launch_counts_by_index(const PlanPtrs &pl, long long n, unsigned *counts_idx, cudaStream_t stream);
// Sorted deposit, second part, per run of equal buffer cells (uniq/lens/offs
// from encode_runs and scan_lengths; nruns on the device): the run's stored
// pair values added in list order on top of the buffer value; short runs one
// thread each, runs longer than a warp one warp each (queued in longq/nlong).
void launch_segment_sum(const Box &B, double *b, const double *pv, const unsigned long long *nruns,
                        const unsigned *uniq, const unsigned *lens, const unsigned *offs, const unsigned *vals,
                        unsigned *longq, unsigned *nlong, cudaStream_t stream);
void launch_return_sinks(const KParams &P, const Box &S, const Parts &p, const double *G, const PlanPtrs &pl,
                         DevStatus *st, cudaStream_t stream);
// Step 4 from the removals the fused ATOMIC deposit stored (pl.pa): a warp
// per sink, lanes over its kernel cells, the sums reduced across the warp
// (their order is not the canonical one; the ATOMIC mode has no bit-exact
// contract).
void launch_return_sinks_stored(const KParams &P, const Box &S, const Parts &p, const PlanPtrs &pl, DevStatus *st,
                                cudaStream_t stream);

void launch_backward_fb(const KParams &P, const Box &S, const double *u, const double *gU, const Parts &p,
                        const PlanPtrs &pl, const unsigned char *pass, const double *G, double *gout,
                        cudaStream_t stream);
void launch_pass_mask(const Box &S, const double *u, const Box &B, const double *b, unsigned char *pass,
                      cudaStream_t stream);
void launch_zero(const Box &B, double *b, cudaStream_t stream);
void launch_fold(const Box &B, double *b, cudaStream_t stream);
// Sink creation (Sec. 3.1.2): flags[v] = 1 for valid cells that qualify, then
// the sinks written at their exclusive-scan positions (count -> *count).
void launch_create_flags(const KParams &P, const Box &S, const double *u, const Box &B, const double *b,
                         unsigned *flags, cudaStream_t stream);
void launch_create_apply(const KParams &P, const Box &S, double *u, const unsigned *flags,
                         const unsigned long long *pos, long long cap, double *x, double *y, double *z, double *m,
                         double *px, double *py, double *pz, long long *count, cudaStream_t stream);
// Auxiliary fields at fixed specific value under accretion (before Step 5).
void launch_apply_extra(const KParams &P, const Box &S, const double *u, const Box &B, const double *b, double *X,
                        int nx, long long xs, cudaStream_t stream);
// App. A.1 rounding of every buffer cell with its error bound E (margin M).
void launch_round(const Box &B, double *b, const double *E, int M, cudaStream_t stream);
// Step 1 for sinks, second half of the scratch form: buffer += s (1, p/rho,
// E/rho) per buffer cell, the factors of its owner cell's D record.
void launch_sink_spread(const Box &S, const Box &B, double *b, const double *scr, const double *drec,
                        cudaStream_t stream);
void launch_sink_aux(const KParams &P, const Box &S, const double *u, double *grec, double *gcs, double *drec,
                     double *dtr, double *deta, cudaStream_t stream);
// Steps 3 + 5 for sinks: eta per valid cell (into deta, for Step 4)
// and U += eta Delta U^sum, in one pass.
void launch_sink_eta_apply(const KParams &P, const Box &S, double *u, const Box &B, const double *b, const double *dtr,
                           double *deta, double *eta_out, DevStatus *st, cudaStream_t stream);
void launch_apply_fb_stream(const Box &S, double *u, const Box &B, const double *b, double *eta_out, DevStatus *st,
                            cudaStream_t stream);
// Steps 3 + 5 without a plan workspace: feedback (FP64 limiter per cell) or
// the particle-mesh kind (eta = 1).
void launch_apply(const KParams &P, const Box &S, double *u, const Box &B, const double *b, double *eta_out,
                  DevStatus *st, cudaStream_t stream);

// CUB primitives, in pmp_sort.cu
size_t cub_temp_bytes(long long n, long long max_pairs, bool sorted);
size_t scan_temp_bytes(long long n);
// Sorts the processing-order keys on bits [0, end_bit): the Morton codes of a
// box whose largest extent needs b bits (b <= 10 after the shift) fill bits
// [0, 3b).  Invalid particles (all-ones keys) then sort among the last
// cell's particles; where they fall in the order does not matter, as they
// have no kernel cells.
cudaError_t sort_host_keys(void *temp, size_t temp_bytes, const unsigned *kin, unsigned *kout, const unsigned *vin,
                           unsigned *vout, long long n, int end_bit, cudaStream_t stream);
cudaError_t scan_counts(void *temp, size_t temp_bytes, const unsigned *counts, unsigned long long *offsets,
                        long long n, cudaStream_t stream);
cudaError_t sort_pairs(void *temp, size_t temp_bytes, const unsigned *kin, unsigned *kout, const unsigned *vin,
                       unsigned *vout, long long n, int end_bit, cudaStream_t stream);
// Runs of equal sorted keys: unique keys, run lengths and their count; the
// exclusive sum of the lengths gives each run's first pair.
cudaError_t encode_runs(void *temp, size_t temp_bytes, const unsigned *keys, unsigned *uniq, unsigned *lens,
                        unsigned long long *nruns, long long n, cudaStream_t stream);
cudaError_t scan_lengths(void *temp, size_t temp_bytes, const unsigned *lens, unsigned *offs, long long n,
                         cudaStream_t stream);

}  // namespace pmp
