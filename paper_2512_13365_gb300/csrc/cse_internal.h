// Internal declarations shared by the kernels and the C-ABI host code of the
// GB300 CSE library.  Not part of the public interface (include/cse.h).
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "cse.h"

// A loaded scheme: per matrix the raw rows, the packed columns, the initial
// candidate list and (A_naive, initial candidate count), all on the device.
struct cse_scheme {
    int n_mats = 0;
    int rows[CSE_MAX_MATS], cols[CSE_MAX_MATS], W[CSE_MAX_MATS], mmax[CSE_MAX_MATS];
    int8_t* d_raw[CSE_MAX_MATS];
    uint2* d_pn0[CSE_MAX_MATS];
    uint32_t* d_cand0[CSE_MAX_MATS];
    int32_t* d_meta0[CSE_MAX_MATS];
    void* d_block = nullptr;
    uint64_t input_hash = 0;  // FNV-1a over every matrix's dimensions and entries (checkpoints record it)
};

namespace cse {

// Strategy indices, in the order of the weights of cse_strategy_mix.
enum Strategy : int { ST_GI = 0, ST_GA = 1, ST_GR = 2, ST_WR = 3, ST_MIX = 4, ST_G = 5, ST_GP = 6, ST_N = 7 };

// Purposes of the Philox draws (third counter word, bits 20..23).
//   RUN    at a run start: lane 0 strategy, 1 alpha, 2 beta, 3 share coin
//   SHAREK prefix length of a shared start (lane 0)
//   STEP   per step, when the strategy draws: lane 0 mix, 1 gr, 2 ga, 3 wr
//   GI     Greedy-Intersections coins of one candidate (extra_lo = its key)
enum Purpose : uint32_t { PU_RUN = 0, PU_SHAREK = 1, PU_STEP = 2, PU_GI = 3, PU_GIS = 4 };

// Per-process state header, in 32-bit words at the start of the process's
// state region in global memory.
enum Hdr : int {
    H_NCOLS = 0, H_NF, H_M, H_COST, H_STRAT, H_A, H_B, H_ENDED, H_RUNS, H_SUBSTEPS,
    H_BEST_COST, H_BEST_LEN, H_TRAJ_LO, H_TRAJ_HI, H_OPS_LO, H_OPS_HI, H_BEST_STRAT, H_MOPS_LO, H_MOPS_HI,
    H_WORDS = 20
};

constexpr int kMaxW = 8;          // 32-bit words per column (256 rows)
constexpr int kMaxCap = 512;      // column capacity
constexpr uint64_t kFnv0 = 0xCBF29CE484222325ull;

// Shared-memory carve-up of one process (one warp), in bytes.
struct WarpLayout {
    int32_t off_cold, off_pn, off_cand, off_f, off_aw, off_poslo, off_hs, off_he, off_base, off_lc;
    int32_t off_pb, off_g, off_pln;  // HBM path: Greedy-Intersections bit-planes
    int32_t off_rec;                 // HBM path: per-variable records (VarRec)
    int32_t off_bv;                  // HBM path: the variable of each 64-position block
    int32_t per_warp;
};

// HBM path: a variable's Greedy-Intersections adjacency in one 16-byte
// record (one sector per variable instead of one per field): its hi-block
// [hs, he) of the list, its running lo rank, its list base, its plane base,
// its lo count and the sum g of the weights (c - 1) of its list.
struct VarRec {
    uint16_t hs, he, lc, vb, pb, lct;
    uint32_t g;
};

// One matrix of one search, as the kernels see it.
struct DevMat {
    const uint2* pn0;        // original columns [nx][W]: x = rows with +1, y = rows with -1
    const uint32_t* cand0;   // initial candidate list, canonical order
    const int32_t* meta0;    // [0] A_naive of the input, [1] initial candidate count
    int32_t rows, nx, W, cap, mmax;  // W: words per column of the kernel (>= wn)
    int32_t wn;              // words per column of the matrix itself, ceil(rows / 32): the
                             // op counts use it, so a wider kernel counts the same ops
    int32_t mat_index;       // index of the matrix within its search (Philox counter)
    int32_t n_proc;
    int32_t search;          // index into the DevSearch array
    int32_t unit_base;       // first work unit of this matrix in its launch
    int32_t state_words;     // 32-bit words per process state region
    uint32_t* state;         // [n_proc][state_words]
    int32_t* best_list;      // [n_proc][cap]
    int32_t* snap;           // [cap]: published best prefix source
    int32_t* snap_meta;      // [0] cost (INT32_MAX = none), [1] length
    unsigned long long* round_min;  // (best cost << 32 | process), min over the round
    int32_t* result;         // [cap] best list of the search
    int32_t* result_meta;    // [0] cost, [1] length
    unsigned long long* counters;   // [0] algorithmic ops, [1] substitution steps,
                                    // [2] process-steps (iteration mode), [3] method ops,
                                    // [4] process-rounds on the process-per-CTA engine,
                                    // [5] process-rounds on the HBM warp engine
    int32_t* curve;          // [kCurvePoints]: lowest best Cost after each round (-1: not run)
    int32_t proc_offset;     // global index of this matrix's first process (a shard of a search
                             // split across ranks; 0 otherwise): draws and round keys use it
    const int32_t* ext_list; // a shard: the round winner's best list when another rank owns it
    const int32_t* ext_len;  //   (uploaded by the host before the share kernel), and its length
    WarpLayout gml;          // layout of the working arrays inside a state region
                             // (HBM path only; fixed for the life of the search)
};

struct DevSearch {
    uint64_t seed;
    uint32_t w[ST_N];
    uint32_t wsum;
    int32_t budget, interval;  // interval 0: iteration mode, budget = max iterations
    int32_t patience;        // iteration mode: stop after this many iterations
                             // without improvement of the total (0: never)
    uint64_t share_thr;      // draw < share_thr => copy a prefix of the snapshot
    int32_t* clock;          // first step of the next round (iteration mode: the
                             // next iteration)
    int32_t* conv;           // iteration mode: [0] iterations without
                             // improvement, [1] converged (the patience rule
                             // ended the search), [2] best total, [3]
                             // iterations run
    const int32_t* mat_pos;  // positions of this search's matrices in the DevMat array
    int32_t n_mats;
    int32_t* status;         // nonzero: a device-side consistency check failed
    int32_t trace;           // record the trajectory hash (CSE_FLAG_TRACE)
    int32_t gi_shared;       // Greedy-Intersections with shared coins (CSE_FLAG_GI_SHARED_COINS)
};

// Process-per-CTA engine (large matrices): one CTA of kCtaThreads threads
// runs one process at a time with the process's working arrays in the CTA's
// shared memory.  A process whose candidate list or Greedy-Intersections
// planes outgrow the capacities below leaves the round unfinished and is
// redone, from its round-start state, by the one-warp-per-process HBM engine
// (round_kernel<W, true, false>), so results never depend on the capacities.
constexpr int kCtaWarps = 16;                      // the widest CTA: 16 warps per process
constexpr int kCtaThreads = 32 * kCtaWarps;
constexpr int kCtaSeg = 12;                        // list entries per lane held in registers
constexpr int kCtaListMax = 32 * kCtaSeg * kCtaWarps;  // 6144: the largest list capacity
constexpr int kCtaMinList = 2048;  // default: shorter lists of a run under way go to the warp engine

struct CtaLayout {
    int32_t off_cold, off_sh, off_pn, off_cand, off_pl, off_aw, off_hs, off_he, off_vb, off_pb, off_lct, off_g;
    int32_t off_lcw, off_f, off_pln;
    int32_t ms;       // candidate capacity (entries)
    int32_t pln_cap;  // Greedy-Intersections plane capacity (64-bit words)
    int32_t min_m;    // a round whose run is under way with fewer candidates runs on the warp engine
    int32_t nw;       // warps per process (CTA): 16 (two CTAs per SM) or 8 (three or four)
    int32_t bytes;    // dynamic shared memory per CTA
};

// planes: the HBM-path layout (weight bit-planes instead of weight bytes).
WarpLayout make_layout(int W, int cap, int mmax, bool planes = false);
// The process-per-CTA layout of a class of matrices; list_cap 0 = automatic
// (the largest that lets two CTAs share an SM).  bytes = 0 if no useful
// layout fits (the class then runs on the warp engine).
CtaLayout make_cta_layout(int W, int cap, int mmax, int list_cap, int min_list, int smem_per_block, int nw = 16);
int state_words(int W, int cap, int mmax);
int state_words_gm(const WarpLayout& L);

// Rounds recorded in a matrix's best-Cost curve.
constexpr int kCurvePoints = 4096;

// A process whose shared-memory slice would exceed this many bytes runs on
// its HBM state region instead (round_kernel<W, true>).
constexpr int kSmemPerWarpLimit = 24 * 1024;

// Launchers (cse_kernels.cu).  All enqueue on `stream` and return the
// launch error, if any.
cudaError_t launch_ingest(const int8_t* raw, int rows, int nx, int W, uint2* pn0, uint32_t* cand0,
                          int32_t* meta0, int mmax, cudaStream_t stream);
// gs: the engine variant with shared Greedy-Intersections coins.
// work: the launch's work counter (zero at launch; the share kernel resets it).
cudaError_t launch_round(int W, bool gm, bool gs, const DevMat* mats, int n_mats, const DevSearch* searches,
                         int total_units, int* work, const WarpLayout& L, int procs_per_cta,
                         cudaStream_t stream);
// The warp engine of the HBM path over a list of units: unit_list[0 ..
// *unit_count) (device memory).
cudaError_t launch_round_list(int W, const DevMat* mats, int n_mats, const DevSearch* searches, int max_units,
                              const int* unit_list, const int* unit_count, int* work, int procs_per_cta,
                              cudaStream_t stream);
cudaError_t launch_round_gs(int W, bool gm, const DevMat* mats, int n_mats, const DevSearch* searches,
                            int total_units, int* work, const WarpLayout& L, int procs_per_cta, cudaStream_t stream,
                            bool prepare_only);
// Also zeroes the n_work (<= 128) work counters of the round kernels.
cudaError_t launch_share(const DevMat* mats, const DevSearch* searches, int n_searches, int* work, int n_work,
                         cudaStream_t stream);
cudaError_t launch_brent(const int8_t* U, const int8_t* V, const int8_t* W, int m, int n, int p, int r,
                         unsigned long long* bad, cudaStream_t stream);
// ctr and out: device arrays of 4 n uint32, 16-byte aligned.
cudaError_t launch_philox(const uint32_t* ctr, long long n, uint64_t seed, uint32_t* out, cudaStream_t stream);
// Sets the launch attributes of a round kernel (call outside stream capture).
cudaError_t prepare_round(int W, bool gm, bool gs, const WarpLayout& L, int procs_per_cta);
// The process-per-CTA engine of a class of large matrices, then the warp
// engine over the processes it handed back.  work3: [0] the CTA engine's work
// counter, [1] the redo launch's work counter, [2] the number of processes
// handed back (all zero at launch; the share kernel resets them).  redo_list:
// room for total_units entries.
cudaError_t launch_round_cta(int W, const DevMat* mats, int n_mats, const DevSearch* searches, int total_units,
                             int* work3, int* redo_list, const CtaLayout& CL, int redo_ppc, cudaStream_t stream);
cudaError_t prepare_round_cta(int W, const CtaLayout& CL, int redo_ppc);
// A whole batch in one persistent cooperative launch (matrices of at most 2
// words per column on the shared-memory engine, step clock): work holds one
// zeroed counter per round, bar two zeroed words, *status 0 (1 after a grid
// barrier gave up after max_spin polls).
cudaError_t launch_batch_persistent(const DevMat* mats, int n_mats, const DevSearch* searches, int n_searches,
                                    int total_units, int rounds, int* work, unsigned* bar, int* status,
                                    unsigned long long max_spin, const WarpLayout& L, int ppc, cudaStream_t stream,
                                    bool prepare_only);
int max_smem_per_block();

// Records the calling thread's error message (cse_last_error) and returns code.
int set_error(int code, const std::string& msg);

}  // namespace cse
