// launch.h -- host-side launchers of the device passes (internal).
#pragma once
#include "dev.cuh"

#include <vector>

namespace vbmc {

// FP64 base pass, tables and screen constants for nq queries (d_qs on device).
// max_sr: max over queries of s * R.
void launch_prologue(const NetView& net, QueryView* d_qs, int nq, int max_sr, cudaStream_t st);

// Shape class of the FP32 SIMT screen for a net (0: unsupported).
int simt_variant(const NetView& net);

// FP32 SIMT screen. Range mode (gather == nullptr): tiles of each query are
// numbered tile_prefix[q] .. tile_prefix[q+1]-1, n_tiles in total, taken from
// the claim counter when one is given (zeroed here; in order, under the time
// budget: see claim_tile). Gather mode: the points are gather[0 ..
// *gather_count). Points the FP32 bound cannot decide go to `out`.
void launch_screen_simt(const NetView& net, const QueryView* d_qs, int nq,
                        const unsigned long long* d_tile_prefix, unsigned long long n_tiles,
                        const QEntry* gather, const unsigned long long* gather_count,
                        unsigned long long gather_cap, Queue out, int out_level, int n_sm,
                        cudaStream_t st, unsigned long long* claim = nullptr);

// Points per tile of the SIMT screen for this net (its range-pass variant).
int simt_tile_points(const NetView& net);

// The FP32 pass for small nets (every layer at most 32 neurons, one thread per
// point): used for single-query calls; its tiles hold small_tile_points().
bool small_supported(const NetView& net);
int small_tile_points();
void launch_small(const NetView& net, const QueryView* d_qs, const unsigned long long* tp,
                  unsigned long long n_tiles, const QEntry* gather, const unsigned long long* gc,
                  unsigned long long gcap, Queue out, int level, int n_sm, cudaStream_t st);

// FP32 pass variants 1..kSimtVariants: widest layer held, points per tile, shared memory.
constexpr int kSimtVariants = 6;
int simt_variant_width(int var);
int simt_variant_default(const NetView& net);
int simt_variant_points(int var);
size_t simt_variant_smem(int var);

// FP64 pass: gather mode over a queue, or range mode over [lo, hi) of query 0
// when gather == nullptr.
void launch_fp64(const NetView& net, const QueryView* d_qs, int nq, const QEntry* gather,
                 const unsigned long long* gather_count, unsigned long long gather_cap,
                 unsigned long long range_lo, unsigned long long range_hi, int n_sm,
                 cudaStream_t st);

// FP64 margin of point t of query 0 into *d_out.
void launch_margin64(const NetView& net, const QueryView* d_qs, unsigned long long t, double* d_out,
                     cudaStream_t st);

// Stamp each query's time-to-verdict after the last pass.
void launch_stamp_final(QueryView* d_qs, int nq, cudaStream_t st);

// Single prologue steps (the allocation-free entry point runs these directly).
void launch_pro_init(const NetView& net, QueryView* d_qs, int nq, cudaStream_t st);
void launch_pro_layer(const NetView& net, QueryView* d_qs, int nq, int l, cudaStream_t st);

// Upper bound of the spectral norm of the row-major m x n matrix A (host data;
// the squarings run on the current device).
double spectral_bound(const std::vector<double>& A, int m, int n);

// Double-float pass (FP32 pairs on CUDA cores) over a queue; points it cannot
// decide go to `out`.
void launch_df(const NetView& net, const QueryView* d_qs, int nq, const QEntry* gather,
               const unsigned long long* gather_count, unsigned long long gather_cap, Queue out,
               int out_level, int n_sm, cudaStream_t st);

// Adversarial points of each of n_tiles contiguous tiles of [0, n) (tiles of
// ceil(n / n_tiles) points) from a verdict bitmap, into d_counts[n_tiles].
void launch_tile_counts(const uint32_t* d_bitmap, unsigned long long n, int n_tiles,
                        unsigned long long* d_counts, cudaStream_t st);

}  // namespace vbmc
