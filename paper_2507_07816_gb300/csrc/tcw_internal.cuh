// tcw_internal.cuh -- shared declarations of the sm_103a track-statistic library.
//
// Method (arXiv:2507.07816): Eq. 1 track, Eq. 2 Doppler factor, nearest-bin
// lookup of the normalized power, weighted sum over segments (Sec. 2) and the
// critical ratio of Eq. 4.  The kernels are organised around one exact
// reformulation of the bin decision:
//
//   a sky s lands above the boundary between bins K and K+1 (frequency
//   c_K = f_min + (K + 1/2) df) iff  fhat >= c_K  iff  v.nhat/c >= c_K/f - 1.
//
// The left side depends on (detector, segment, sky) only, the right side on
// (template, segment, K) only.  Both are rounded once to an integer grid of
// step q (the left with floor, the right with round), so the decision becomes
// one int32 compare per lookup and differs from the exact real decision only
// when the track lies within F*q/2 bins of the boundary, F = f/df.  The host
// picks q so that F*q/2 stays below 0.75 * 2^-30 bins.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tcw.h"

namespace tcw {

constexpr double kLightSpeed = 299792458.0;  // m/s
constexpr int kMaxDet = 8;

// Bin window of the group kernel, relative to a per-(template, segment) base
// bin: candidates base + m for m in [kMLo, kMHi]; threshold i separates
// base + kMLo + i from base + kMLo + i + 1.
constexpr int kMLo = -4;
constexpr int kMHi = 4;
constexpr int kNThr = kMHi - kMLo;  // 8 thresholds

// Precomputed per (template, segment): 96 bytes, lives in shared memory.
//   F, Cm  fp32 estimates that choose the candidate bin pair: for a sky group
//          whose mean Doppler factor is g, the pair starts at
//          base + n0 with n0 = round(F*g + Cm)   (Cm = (f - f_min)/df - base - 1/2),
//          computed as zb = bits(F*g + Cm + kMagic), n0 = zb - kMagicBits
//   tha    shared address of th[] minus 4*(kMagicBits + kMLo): threshold of
//          the pair is at tha + 4*zb
//   cls    kEntryNone / kEntryInside / kEntryEdge
//   wa[d], wf[d]  group-uniform path: window address (power of bin base + n0
//          at wa[d] + elem*zb) and weight; for entries that are not wholly in
//          the band wa points at a zero window and wf = 0
//   kb     base - kMagicBits, so that base + n0 = kb + zb
//   xa[d], we[d]  per-sky path: the staged power window of detector d and the
//          lookup weight w_{d,j} (f(t_j)/f0)^p (Eq. 3 factor, 1 when p = 0)
//   th[i]  round((c_K/f - 1)/q) with c_K = f_min + (K + 1/2) df, K = base + kMLo + i
struct __align__(16) TrackEntry {
  float F;
  float Cm;
  uint32_t tha;
  int cls;
  uint32_t wa[2];
  float wf[2];
  int kb;
  uint32_t xa[2];
  int pad0;
  float we[2];
  float pad1[2];
  int th[kNThr];
};
static_assert(sizeof(TrackEntry) == 96, "track entry layout");

constexpr int kEntryNone = 0;    // segment before T0, or every candidate bin outside the band
constexpr int kEntryInside = 1;  // every candidate bin inside the band
constexpr int kEntryEdge = 2;    // candidates straddle a band edge
constexpr float kMagic = 12582912.0f;     // 1.5 * 2^23: x + kMagic rounds x to an integer
constexpr int kMagicBits = 0x4B400000;    // bit pattern of kMagic

// One event of a search: its spectrogram, segment times, Doppler blocks, tile
// anchors and outputs.  A plain search is a batch of one event.
struct EventDesc {
  const void* rho;         // [D][n_seg][pitch] float or half, 16-byte aligned base
  const float* weights;    // [D][n_seg]
  const double* t_mid;     // [n_seg]
  const int32_t* blk;      // Doppler blocks [Spad / (16 lanes)][n_seg][D][block_words(lanes)]
  const double* anchors;   // [Bpad][n_tiles][2]: 1/f and 1/(tau + t_a - T0) at each tile's
                           // anchor t_a; read only when nterms > 0
  const double* f0;        // the event's sorted bank [Bpad] (events may share one)
  const double* tau;
  const double* nbr;
  int Bpad;                // templates of the bank arrays (a multiple of every pass)
  float* psi;              // [Spad][Bpad]
  float* S_out;            // optional [Spad][Bpad]
  float* W1_out;
  float* W2_out;
  int64_t total_elems;     // D * n_seg * pitch
  double T0;
  int n_seg, n_tiles, S, Spad, NG;
  int bit_pitch;           // words per row of `bits`
  const uint32_t* bits;    // number count: [D][n_seg][bit_pitch] bit k of a row = [rho_k > rho_th];
                           // null for the power statistic
};

// Work item of the group kernel: one sky chunk of 16 lanes sorted directions
// of one event x `groups` consecutive groups of 512 / lanes sorted templates.
//   x = event, y = sky chunk, z = first sorted template, w = groups
// CTA i runs items [cta_items[i], cta_items[i + 1]) in order.
struct GroupParams {
  const EventDesc* events;
  const int4* items;
  const int* cta_items;    // [gridDim.x + 1]
  int64_t n_bin;           // bins per row that belong to the band
  int64_t pitch;           // elements between rows (>= n_bin)
  int n_det;               // <= kMaxStageDet
  double f_min, df, inv_q;
  int nterms;              // binomial-series length for the track; 0 = pow per entry
  int tile_shift;          // tiles of 2^tile_shift segments: anchors and fp32 partial sums
  int amp_power;           // weights times (f(t_j)/f0)^amp_power (Eq. 3); 0 = none
  double nc_q;             // number count: q = exp(-rho_th), <s> = q W1, sigma^2 = q(1-q) W2;
                           // 0 = power (<s> = W1, sigma^2 = W2).  Needs every event's bits.
  int track_bins;          // 2: each lookup sums the bins floor(x), floor(x) + 1 (staged as fp32
                           // pair sums; <s> and sigma^2 doubled); otherwise the nearest bin
  int map_half;            // the events' maps are fp16 (read by the two-bin producers)
  int B;                   // templates of the bank (recording only)
  int lanes;               // sky groups per chunk: 16, 32 or 64
  float2* dev;             // scratch [gridDim.x][kPassUnits * 16]: per-sky weight sums at band edges
  int32_t* rec;            // optional [S][B][D][Nseg], caller order (single-event searches)
  const int32_t* bank_perm;  // sorted -> caller template index
  const int32_t* sky_perm;   // sorted -> caller sky index (event 0)
  unsigned long long* n_general;
  int* err;                // bit 0: window, bit 1: a bounded wait ran out
};

// Tile anchors of one event for every sorted template.
struct AnchorParams {
  const double* t_mid;
  const double* f0;
  const double* tau;
  const double* nbr;
  double T0;
  int n_seg, n_tiles, tile_shift, Bpad;
  double* anchors;         // [Bpad][n_tiles][2]
  int chain;               // 1: each run of kAnchorRun tiles takes pow at its first anchor and the
                           // binomial series from anchor to anchor after it; 0: pow at every anchor
};
constexpr int kAnchorRun = 16;     // anchors per pow in the chained form
constexpr int kAnchorTerms = 20;   // binomial-series terms of one anchor-to-anchor step
// 1 when the anchor-to-anchor steps of these segment times allow the chained
// form: u'/u - 1 <= 0.1 and the series' remainder below 2^-56 relative.
int anchor_chain_for(const double* t_mid, int64_t n_seg, double T0, int tile, double tau_min, double r_max);

struct LookupParams {
  const void* rho;
  int64_t n_bin;
  int n_det;
  int n_seg;
  const float* weights;
  const double* t_mid;
  const double* vel;       // [D][Nseg][3]
  const double* nhat;      // sorted sky [Spad][3]
  const double* f0;
  const double* tau;
  const double* nbr;
  double T0, f_min, df;
  int amp_power;           // weights times (f(t_j)/f0)^amp_power (Eq. 3); 0 = none
  int number_count;        // 1: nu = [rho > rho_th] in place of rho, Psi with q = exp(-rho_th)
  double rho_th;
  int track_bins;          // 2: the bins floor(x), floor(x) + 1 per lookup; otherwise the nearest
  int B, Bpad, S, Spad;
  float* psi;
  float* S_out;
  float* W1_out;
  float* W2_out;
  int32_t* rec;
  const int32_t* bank_perm;
  const int32_t* sky_perm;
};

// One Doppler block per (sky chunk of 16 L sorted skies, segment, detector),
// L = lanes (sky groups) per chunk:
//   words [0, 16 L): floor(v.nhat/c / q) of sky 16 g + k at 16 g + k
//   words [16 L + 4 g, 16 L + 4 g + 4): sky group g's fp32 mid-range of v.nhat/c
//                    (bits), the smallest and the largest of its 16 grid values, 0
// so that one bulk copy moves a chunk's segment for every detector.
__host__ __device__ constexpr int block_words(int lanes) { return 20 * lanes; }

struct DopplerParams {
  const double* vel;       // [D][Nseg][3]
  const double* nhat;      // [Spad][3] sorted
  int n_det, n_seg, Spad, NG, group;
  int lanes;               // sky groups per chunk (16, 32 or 64)
  double inv_q;
  int32_t* blk;            // [Spad / (16 lanes)][Nseg][D][block_words(lanes)]
  unsigned* spread_max;    // float bits of max (hi - lo) of v.nhat/c over the groups
};

constexpr int kMaxSeriesTerms = 20;   // longest track series (more: pow per entry)
constexpr int kMaxStageDet = 2;          // detectors the group kernel stages in shared memory
constexpr int kTileShift = 5;           // default tile: 32 segments

// dynamic shared memory of the group kernel for D detectors
size_t group_smem_bytes(int n_det, int lanes);
cudaError_t launch_anchors(const AnchorParams& p, cudaStream_t st);
// per-CTA scratch of the group kernel, in float2 elements
size_t group_dev_elems(int grid);

// ---------------------------------------------------------------------------
// Learned sky triage (tcw_triage.cu)
// ---------------------------------------------------------------------------
constexpr int kTriageBins = 128;  // histogram bins = MLP inputs
constexpr int kMlpIn = 128, kMlpH = 256;
// packed fp32 parameters: W1 [128][256] | b1 [256] | W2 [256][256] | b2 [256] | w3 [256] | b3
constexpr int64_t kThW1 = 0, kThB1 = kThW1 + kMlpIn * kMlpH, kThW2 = kThB1 + kMlpH,
                  kThB2 = kThW2 + kMlpH * kMlpH, kThW3 = kThB2 + kMlpH, kThB3 = kThW3 + kMlpH,
                  kMlpParams = kThB3 + 1;
// bfloat16 weights read by the forward pass: W1 | W2 | w3
constexpr int64_t kWbfW1 = 0, kWbfW2 = kWbfW1 + kMlpIn * kMlpH, kWbfW3 = kWbfW2 + kMlpH * kMlpH,
                  kMlpWeights = kWbfW3 + kMlpH;
// position of packed parameter i in the bfloat16 weights, or -1 for a bias
__host__ __device__ inline int64_t mlp_weight_index(int64_t i) {
  if (i >= kThW1 && i < kThB1) return kWbfW1 + (i - kThW1);
  if (i >= kThW2 && i < kThB2) return kWbfW2 + (i - kThW2);
  if (i >= kThW3 && i < kThB3) return kWbfW3 + (i - kThW3);
  return -1;
}

struct PatchDopplerParams {
  const double* vel;        // [D][n_seg_full][3]
  const double* nhat;       // sorted sky [S][3]
  int n_det, n_seg, S, patch_size, P;   // n_seg: coarse segments (segment j' is j' stride)
  int stride, n_seg_full;
  float* dop;               // [D][n_seg][P]
};

struct CoarseParams {
  const void* rho;          // [D][n_seg_full][n_bin]
  int64_t n_bin;
  int n_det, n_seg;         // n_seg: coarse segments; coarse segment j' is segment j' stride
  int stride, n_seg_full;
  const float* weights;     // [D][n_seg_full]
  const double* t_mid;      // [n_seg] times of the coarse segments
  double T0, f_min, df;
  const float* dop;         // [D][n_seg][P]
  int P;
  const double* f0;         // sorted bank [Bpad]
  const double* tau;
  const double* nbr;
  int B, Bpad;              // Bpad a multiple of 4
  const double* anchors;    // [Bpad][n_tiles][2] at 32-segment tiles, or null when nterms == 0
  int n_tiles, nterms;
  float lo, hi;             // histogram range of Psi
  float* psi;               // optional [P][Bpad]
  unsigned* hist;           // [P][128], zero at launch
  float* feat;              // [P][128] log(1 + count)
  int parts;                // segment ranges the tiles are split into (set by launch_coarse)
  double* part_acc;         // [parts][P][Bpad][3] partial S, W1, W2 when parts > 1 (size from coarse_part_elems)
};
// Elements of CoarseParams::part_acc that launch_coarse may use.
size_t coarse_part_elems(int P, int Bpad);

cudaError_t launch_patch_doppler(const PatchDopplerParams& p, cudaStream_t st);
cudaError_t launch_coarse(const CoarseParams& p, bool half, cudaStream_t st);

// Coarse pass, sweep form.  Where the representatives' Doppler factors are
// non-decreasing in patch order at a (detector, segment), the bin of a
// (template, segment, detector) lookup is a non-decreasing step function of
// the representative, so one thread per template gathers the first
// representative's bin and records each step's power difference in a
// per-template difference array; a prefix sum over the representatives
// gives every S (Eq. 4 numerator).  The other (detector, segment) pairs (two
// representatives' factors cross there) take every representative's own bin.
constexpr int kSweepThreads = 256;
constexpr int kSweepMaxPatches = 128;   // shared memory: (P + 1) x kSweepThreads floats
constexpr int kSweepMaxTerms = 24;      // FP64 binomial terms of the anchor-to-anchor step

struct SweepDopplerParams {
  const double* vel;        // [D][n_seg_full][3]
  const double* nhat;       // sorted sky [S][3]
  int n_det, n_seg, S, patch_size, P, P2;   // P2: power of two >= P
  int stride, n_seg_full;
  float* dop;               // [D][n_seg][P2] v.nhat/c of each representative, +inf beyond P
  int* unsorted;            // [D][n_seg], zero at launch: set to 1 where the factor decreases
                            // from one representative to the next
};

struct CoarseSweepParams {
  const void* rho;          // [D][n_seg_full][n_bin]
  const void* rho_i;        // two detectors: [n_seg][n_bin][2], the coarse segments interleaved
  int64_t n_bin;
  int n_det, n_seg, stride, n_seg_full;   // n_seg: coarse segments
  const float* weights;     // [D][n_seg_full]
  const float4* seg;        // [n_seg] {dt hi, dt lo, dt^2 hi, dt^2 lo}, dt = t - anchor time of the
                            // segment's tile (fp32 pairs of the FP64 values); dt hi = NaN where t < T0
  const double* ta;         // [n_tiles] anchor times, NaN for tiles without a segment at or after T0
  int tile_shift, n_tiles, nt64;
  double T0, f_min, df;
  double inv_df, xmin;      // 1/df and f_min/df
  const float* dop;         // [D][n_seg][P2] from SweepDopplerParams
  const int* unsorted;      // [D][n_seg] from SweepDopplerParams: those lookups take every
                            // representative one by one
  int P, P2;
  const double* f0;         // sorted bank [Bpad]
  const double* tau;
  const double* nbr;
  int B, Bpad;
  double* coef64;           // [nt64 + 3][Bpad] scratch: binomial coefficients C(e, k) of each
                            // template, then 1/tau, e and C(e, 2)
  double* w2edge;           // [P + 1][Bpad] zero at launch: W2 steps of band-edge lookups
  int* nedge;               // [P + 1][Bpad] zero at launch: valid-lookup count steps of them
  int parts;                // segment ranges per template (a multiple of 64 segments each)
  float* part_S;            // [parts][P][Bpad] when parts > 1: S - W1 per range
  float* part_W2;           // [parts][Bpad] when parts > 1: W2 of in-band lookups per range
  float lo, hi;
  float* psi;               // optional [P][Bpad]
  unsigned* hist;           // [P][128], zero at launch
  float* feat;              // [P][128] log(1 + count)
};

cudaError_t launch_sweep_doppler(const SweepDopplerParams& p, cudaStream_t st);
cudaError_t launch_interleave(const void* rho, bool half, int64_t n_bin, int n_seg, int stride, int n_seg_full,
                              void* out, cudaStream_t st);
// Template regions of a triaged search: for each listed row r of the coarse
// Psi [P][Bpad] (sorted bank, first B valid), keep[b] = 1 for its M best
// templates by (Psi desc, index asc); rows OR into one keep [B].
cudaError_t launch_region_select(const float* psi, int Bpad, int B, const int* rows, int n_rows, int M,
                                 unsigned char* keep, cudaStream_t st);
// dst[i][:width] = src[idx[min(i, n - 1)]][:width] for i < npad (64-bit elements)
cudaError_t launch_gather_rows(const double* src, const int32_t* idx, int64_t n, int64_t npad, int width,
                               double* dst, cudaStream_t st);
cudaError_t launch_gather_rows(const int32_t* src, const int32_t* idx, int64_t n, int64_t npad, int width,
                               int32_t* dst, cudaStream_t st);
// psi[i] = -inf and idx[i] = -1 for i < n
cudaError_t launch_fill_empty(float* psi, int64_t* idx, int64_t n, cudaStream_t st);
// nc: fp32 terms of the in-tile series beyond the quadratic one (4, 6 or 8)
cudaError_t launch_coarse_sweep(const CoarseSweepParams& p, bool half, int nc, cudaStream_t st);
// Segment ranges per template for the sweep form: the count in [1, 4] whose
// blocks finish soonest on the device's resident slots.
int sweep_parts(const CoarseSweepParams& p, bool half, int nc);
// selected[p] = 1 for the m best patches; a chosen patch suppresses the
// patches within `radius` of it (0 = plain ranking)
cudaError_t launch_rank(const float* score, int P, int m, int radius, int* selected, cudaStream_t st);
cudaError_t mlp_forward(const __nv_bfloat16* wbf, const float* theta, const float* X, int64_t n, float* H1,
                        float* H2, float* y, cudaStream_t st);
// work: 2 * n * 256 floats
cudaError_t mlp_backward(const __nv_bfloat16* wbf, const float* X, int64_t n, const float* H1, const float* H2,
                         const float* dy, float* grad, float* work, cudaStream_t st);
cudaError_t mlp_bce(const float* y, const float* label, int64_t n, float pw, float* loss, float* dy,
                    cudaStream_t st);
cudaError_t mlp_adam(float* theta, float* m, float* v, const float* grad, int64_t step, float lr, float b1,
                     float b2, float eps, __nv_bfloat16* wbf, cudaStream_t st);
cudaError_t mlp_pack(const float* theta, __nv_bfloat16* wbf, cudaStream_t st);

// Host helpers of the group kernel (tcw_persist.cu; the kernel is in tcw_persist.cuh).
// CTAs of a group-kernel launch on the current device: one per SM.
cudaError_t group_grid(int* grid);
// Longest-processing-time-first schedule: items in decreasing cost, each to
// the CTA with the least work so far (ties: lowest CTA, and equal costs keep
// their order).  out = the items grouped by CTA, cta_items = [grid + 1] offsets.
void schedule_items(const std::vector<int4>& items, const std::vector<int64_t>& cost, int grid,
                    std::vector<int4>& out, std::vector<int>& cta_items);
// Length of the binomial series sum_k binom(r, k) delta^k that gives 1/f(t_j)
// from its tile anchor to below 2^-56 relative, for every template (tau >=
// tau_min, r = 1/(n-1) <= r_max) and tile of `tile` segments; 0 when more
// than kMaxSeriesTerms terms would be needed.
int series_terms_for(const double* t_mid, int64_t n_seg, double T0, int tile, double tau_min,
                     double r_max);
inline int ilog2(int v) {
  int r = 0;
  while ((1 << (r + 1)) <= v) ++r;
  return r;
}

// launchers (return cudaError_t of the launch)
cudaError_t launch_doppler(const DopplerParams& p, cudaStream_t st);
// Set the shared-memory attribute of the group-kernel variant (also done by
// launch_group on first use); call before capturing a launch into a graph.
// pw: windows built by the producer (number count or two-bin lookups; fp32 only).
cudaError_t group_prepare(int n_det, int lanes, bool half, bool pw);
// grid = number of CTAs (the length of p.cta_items minus one); one CTA per SM at most.
// Every lookup is weighted by p.events[].weights (times the amplitude factor
// when p.amp_power > 0).
cudaError_t launch_group(const GroupParams& p, int grid, bool half, bool record, cudaStream_t st);
cudaError_t launch_lookup(const LookupParams& p, bool half, bool record, cudaStream_t st);
// A generated template bank (tcw_bank_spec on the device).
struct BankGenParams {
  int kind;                // TCW_BANK_LATTICE or TCW_BANK_RANDOM
  int64_t n_f0, n_tau, n_n;
  double lo[3], hi[3];     // (f0, tau, n) bounds
  uint64_t seed;
};
cudaError_t launch_gen_bank(const BankGenParams& p, int64_t first, int64_t count, int64_t pad_to, double* f0,
                            double* tau, double* nbr, int32_t* perm, cudaStream_t st);
// Templates at the indices at[0 .. count) (device, each inside the bank).
cudaError_t launch_gen_bank_at(const BankGenParams& p, const int64_t* at, int64_t count, double* f0, double* tau,
                               double* nbr, cudaStream_t st);
// Per sky: the first k of the merge of a (ra entries) and b (rb entries, local
// indices + b_base) by (Psi desc, index asc) into o; rows of a and o hold k.
cudaError_t launch_merge_topk(const float* a_psi, const int64_t* a_idx, int ra, const float* b_psi,
                              const int64_t* b_idx, int rb, int64_t b_base, int k, int64_t S, float* o_psi,
                              int64_t* o_idx, cudaStream_t st);
// Number-count bit map: bits[r][w] bit i = [rho[r][32 w + i] > rho_th] (compared
// in double; 0 past n_bin) for rows r < rows, words w < bit_pitch.
int bit_pitch_for(int64_t n_bin);
cudaError_t launch_count_bits(const void* rho, bool half, int64_t rows, int64_t n_bin, int bit_pitch,
                              double rho_th, uint32_t* bits, cudaStream_t st);
cudaError_t launch_topk(const float* psi, int Bpad, int B, int S, int k, const int32_t* bank_perm,
                        const int32_t* sky_perm, float* psi_out, int64_t* idx_out,
                        cudaStream_t st);
cudaError_t launch_unpermute(const float* src, int Spad, int Bpad, int S, int B,
                             const int32_t* sky_pos, const int32_t* bank_pos, float* dst,
                             cudaStream_t st);

// group-kernel geometry (shared by the host planner and the kernels): a sky
// chunk is `lanes` groups of kGroupSkies sorted skies (lanes = 16, 32 or 64),
// and one pass of the kernel covers one chunk x 1024 / lanes templates.
constexpr int kGroupSkies = 16;     // skies of one sky group
constexpr int kPassUnits = 1024;    // (template, sky group) units of one pass of the group kernel
constexpr int kBankAlign = 64;      // Bpad is a multiple of every pass's template count
__host__ __device__ constexpr int chunk_skies(int lanes) { return kGroupSkies * lanes; }
__host__ __device__ constexpr int pass_templates(int lanes) { return kPassUnits / lanes; }
inline int padded_skies(int64_t S, int lanes) {
  const int64_t ng = (S + kGroupSkies - 1) / kGroupSkies;
  return (int)((ng + lanes - 1) / lanes) * chunk_skies(lanes);
}
// Relative cost of one padded (template, sky, segment) at each chunk width:
// a narrow chunk computes the track entries of 4x (2x) more templates per
// stage for the same number of lookups (measured on GB300 at 1e4 segments).
inline double lanes_cost(int lanes) { return lanes == 16 ? 1.6 : (lanes == 32 ? 1.25 : 1.0); }
// The chunk width with the lowest padded cost (ties: the widest chunk).
inline int choose_lanes(int64_t S) {
  int best = 64;
  for (int l : {32, 16})
    if (padded_skies(S, l) * lanes_cost(l) < padded_skies(S, best) * lanes_cost(best)) best = l;
  return best;
}
// With the bank and the grid known: a work item is one chunk (16 L skies) x
// bank_chunk passes of 1024 / L templates, 16384 padded sky-templates per pass
// whatever L, so the search takes ceil(items / grid) rounds of items costing
// lanes_cost(L) each.  Few templates give few items at narrow chunks, and a
// wider chunk can then fill more SMs.
inline int choose_lanes(int64_t S, int64_t B, int bank_chunk, int grid) {
  if (B <= 0 || grid <= 0) return choose_lanes(S);
  int best = 0;
  double best_cost = 0;
  for (int l : {64, 32, 16}) {
    const int64_t chunks = padded_skies(S, l) / (16 * l);
    const int64_t groups = (B + pass_templates(l) - 1) / pass_templates(l);
    const int64_t items = chunks * ((groups + bank_chunk - 1) / bank_chunk);
    const double cost = (double)((items + grid - 1) / grid) * bank_chunk * lanes_cost(l);
    if (best == 0 || cost < best_cost) {
      best = l;
      best_cost = cost;
    }
  }
  return best;
}

}  // namespace tcw
