// Kernel-side data structures of libonmf (shared by the kernels and the
// host code that launches them). Layouts in HBM:
//
//   V     F x n  float, column (frame) major, leading dimension ldv.
//   Wcm   F x K  float, column-major: the dictionary W (state).
//   Wrm   F x K  float, row-major copy of W (FP32 path, K-contiguous rows).
//   Wimg  Kp x WLD bf16: W^T padded for the tensor-core path; row k holds
//         column k of W (F values, zero padded to WLD = Fp16 + 8). The +8
//         makes 8 consecutive rows fall in distinct shared-memory banks.
//   Wrow  F x Kp bf16: W row-major (tcgen05 and cluster h-solves).
//   A, B  F x K  double, column-major: the sufficient statistics (Eq. aux_fun).
//   Pg,Qg betap x Fp16: per-frame rows of P = Y/X^2 and Q = 1/X of the
//         current minibatch (float on the FP32 path, bf16 on the mixed path).
//   Hg    FP32 path: betap x Kh float (frame rows); mixed path: Kh x betap
//         bf16 (k rows, frames contiguous).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace onmf {

constexpr int kThreads = 256;  // threads per CTA for every kernel here
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 8;       // frames per h-solve tile (mma.sync and FP32 paths)
constexpr int kTcTile = 16;    // frames per h-solve tile (tcgen05 path)

// PREC_TC: the mixed-precision arithmetic with the tcgen05 (TMEM) h-solve;
// PREC_CL: the same arithmetic with the cluster h-solve (W split by rows
// over the CTAs of a thread-block cluster, 32-frame tiles).
enum Prec : int { PREC_FP32 = 0, PREC_MIXED = 1, PREC_TC = 2, PREC_CL = 3 };

struct Shape {
    int F, K;
    int Fp16;  // F rounded up to 16
    int Kp;    // K rounded up to 16
    int Kh;    // K rounded up to 32 (statistics k-slabs, ld of Hg on FP32)
    int WLD;   // row stride of Wimg (Fp16 + 8)
};

__host__ __device__ inline Shape make_shape(int F, int K) {
    Shape s;
    s.F = F;
    s.K = K;
    s.Fp16 = (F + 15) / 16 * 16;
    s.Kp = (K + 15) / 16 * 16;
    s.Kh = (K + 31) / 32 * 32;
    s.WLD = s.Fp16 + 8;
    return s;
}

// Frame ranges of the tcgen05 statistics of the mma path (onmf_stats_tc.cuh).
constexpr int kMaxRanges = 256;  // completion counters of the ranges, after the barrier word
struct StatsSplit {
    int S;    // frame ranges
    int gps;  // 8-frame groups per range (even: whole 16-frame MMA steps)
};

// Frame ranges of a minibatch of nb frames for a grid of G CTAs and FT
// frequency tiles: FT * S units on about half of the grid (each range is one
// more partial sum for the column pass to add, so fewer, longer ranges),
// with at least one 16-frame step per range.
// S_req > 0 asks for that many ranges instead (onmf_config.stats_ranges).
__host__ __device__ inline StatsSplit stats_split(int nb, int G, int FT, int S_req = 0) {
    const int ng = (nb + 7) / 8;
    int S = S_req > 0 ? S_req : (G / (2 * FT) > 1 ? G / (2 * FT) : 1);
    if (S > kMaxRanges) S = kMaxRanges;
    const int steps = (ng + 1) / 2;
    if (S > steps) S = steps;
    if (S < 1) S = 1;
    int gps = (ng + S - 1) / S;
    gps = (gps + 1) / 2 * 2;
    StatsSplit r;
    r.gps = gps;
    r.S = (ng + gps - 1) / gps;
    return r;
}

// Arguments of the online step kernel (one launch = nmb minibatches).
struct StepArgs {
    Shape s;
    float eps;
    float gamma;
    int n_in;
    int normalize;
    int rho_on_new;
    int acc;  // arithmetic of A and B (ACC_*)
    int stats_ranges;  // frame ranges of the tcgen05 statistics (0: automatic)
    float hpen, hpen_a, wpen;  // penalties (FP32, mma, cluster paths): lambda, a, mu
    // frames
    const float *V;
    long long ldv;
    int nmb;      // minibatches in this launch
    int beta;     // frames per full minibatch
    int nb_last;  // frames in the last minibatch (<= beta)
    double rho_full, rho_last;
    float *H_out;  // optional K x frames (ldh)
    long long ldh;
    const float *H_in;  // warm restarts: start points, K x frames (ldh_in), or NULL
    long long ldh_in;
    // state
    float *Wcm;
    float *Wrm;
    __nv_bfloat16 *Wimg;
    __nv_bfloat16 *Wrow;  // tensor-core path: bf16 W, row f = row f of W (ld Kp)
    float *Wn;
    double *A, *B;
    double *loss_sum;
    float *swpart;  // [K] column sums of the normalized W
    // scratch
    void *Pg, *Qg, *Hg;
    int betap;  // rows of Pg/Qg (and columns of the bf16 Hg)
    float *part;  // mma path: frame-range partial sums of P H^T, Q H^T
    double *loss_part;
    unsigned *bar;  // [0]: grid barrier; [4, 4 + kMaxRanges): frame-range counters
    int *err;
    long long *stamps;  // phase-timing build only (ONMF_PHASE_STAMPS), else NULL
};

// Phase timing (a build option for measurement, ONMF_PHASE_STAMPS): thread 0
// of every CTA writes a time at kStampPts points of each of the first
// kStampMb minibatches of a launch, [minibatch][CTA][point]; points 0-6 are
// the phase boundaries of the online step (%globaltimer, ns), 8-14 the steps
// of a statistics unit (clock64, the CTA's last unit of the minibatch), 7
// and 15 the %globaltimer at the unit's first and last step.
// Points 16-31: the CTA's first h-solve tile of the minibatch (clock64):
// 16 tile start, 17 frames in shared memory and converted, 18 W^T image in
// shared memory, 19 + i end of inner iteration i (up to 10), 29 final ratios
// and loss, 30 P, Q, H rows written, 31 end of step A of iteration 10.
// Points 32-33 (%globaltimer): in the window of the grid barrier before the
// column pass, 32 after the arrival and the column's W, A, B loads, 33
// after the next minibatch's frames are staged; 34-37 (clock64) the steps of that staging;
// 38-39 (%globaltimer) the start and end of the CTA's first h-solve tile;
// 40-44 (clock64) the steps of the CTA's first column of the column pass.
#ifndef ONMF_STAMP_PTS
#define ONMF_STAMP_PTS 48  // points per (minibatch, CTA) record
#endif
constexpr int kStampMb = 128, kStampCtas = 256, kStampPts = ONMF_STAMP_PTS;

// Arguments of the projection / batch h-step kernels (no state update).
struct TileArgs {
    Shape s;
    float eps;
    float gamma;
    int n_in;
    const float *V;
    long long ldv;
    long long n;          // frames
    const float *H_in;    // warm start (K x n, ld ldh_in) or NULL = fresh restart
    long long ldh_in;
    float *H_out;         // K x n (ldh) or NULL
    long long ldh;
    int loss_first;       // loss of the first X (before any h update) only
    int final_pass;       // compute X from the final h: P/Q/Hg rows, the loss unless loss_first
    const float *Wcm;
    const float *Wrm;
    const __nv_bfloat16 *Wimg;
    const __nv_bfloat16 *Wrow;
    const float *swpart;
    void *Pg, *Qg, *Hg;
    long long betap;
    double *loss_part;    // [tiles] or NULL
    int *err;
    float hpen, hpen_a;   // h penalty lambda, a (lambda = 0: none)
};

}  // namespace onmf
