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

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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

// Precomputed per (template, segment): 80 bytes, lives in shared memory.
//   F, Cm  fp32 estimates that choose the candidate bin pair: for a sky group
//          whose mean Doppler factor is g, the pair starts at
//          base + n0 with n0 = round(F*g + Cm)   (Cm = (f - f_min)/df - base - 1/2),
//          computed as zb = bits(F*g + Cm + kMagic), n0 = zb - kMagicBits
//   tha    shared address of th[] minus 4*(kMagicBits + kMLo): threshold of
//          the pair is at tha + 4*zb
//   cls    kEntryNone / kEntryInside / kEntryEdge
//   wa[d]  shared address of detector d's staged power window minus
//          elem*(kMagicBits + woff_d): power of bin base + n0 is at wa[d] + elem*zb
//   kb     base - kMagicBits, so that base + n0 = kb + zb
//   th[i]  round((c_K/f - 1)/q) with c_K = f_min + (K + 1/2) df, K = base + kMLo + i
struct __align__(16) TrackEntry {
  float F;
  float Cm;
  uint32_t tha;
  int cls;
  uint32_t wa[4];
  int kb;
  int pad[3];
  int th[kNThr];
};

constexpr int kEntryNone = 0;    // segment before T0, or every candidate bin outside the band
constexpr int kEntryInside = 1;  // every candidate bin inside the band
constexpr int kEntryEdge = 2;    // candidates straddle a band edge
constexpr float kMagic = 12582912.0f;     // 1.5 * 2^23: x + kMagic rounds x to an integer
constexpr int kMagicBits = 0x4B400000;    // bit pattern of kMagic

struct GroupParams {
  const void* rho;         // [D][Nseg][pitch] float or half, 16-byte aligned base
  int64_t n_bin;           // bins per row that belong to the band
  int64_t pitch;           // elements between rows (>= n_bin)
  int64_t total_elems;     // D * Nseg * pitch
  int n_det;               // <= kMaxStageDet
  int n_seg;
  const float* weights;    // [D][Nseg]
  const double* t_mid;     // [Nseg]
  const int32_t* blk;      // Doppler blocks [NGpad/64][Nseg][D][kBlockWords], see kBlockWords
  const double* f0;        // sorted bank, [Bpad]
  const double* tau;
  const double* nbr;
  double T0, f_min, df, inv_q;
  int nterms;              // binomial-series length for the track; 0 = pow per entry
  const double* anchors;   // [Bpad][n_tiles][2]: 1/f and 1/(tau + t_a - T0) at each tile's
                           // anchor t_a; read only when nterms > 0
  int n_tiles;             // ceil(Nseg / kTileSegments)
  int B, Bpad, S, Spad, NG, NGpad;
  int n_chunks;            // Spad / 1024 sky chunks
  int n_items;             // n_chunks * Bpad / 8 work items; item i runs on CTA i mod grid
  float* psi;              // [Spad][Bpad]
  float* S_out;            // optional [Spad][Bpad]
  float* W1_out;
  float* W2_out;
  float2* dev;             // scratch [Bpad][Spad]: per-sky weight sums at band edges
  int32_t* rec;            // optional [S][B][D][Nseg], caller order
  const int32_t* bank_perm;  // sorted -> caller template index
  const int32_t* sky_perm;   // sorted -> caller sky index
  unsigned long long* n_general;
  int* err;                // bit 0: window, bit 1: a bounded wait ran out
};

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
  int B, Bpad, S, Spad;
  float* psi;
  float* S_out;
  float* W1_out;
  float* W2_out;
  int32_t* rec;
  const int32_t* bank_perm;
  const int32_t* sky_perm;
};

// One Doppler block per (sky chunk of 1024 sorted skies, segment, detector):
//   words [0, 1024): floor(v.nhat/c / q) of sky 16 g + 4 v + k at (v * 64 + g) * 4 + k
//   words [1024, 1088): fp32 mid-range of v.nhat/c over sky group g (bits)
// so that one bulk copy moves a chunk's segment for every detector.
constexpr int kBlockWords = 1088;

struct DopplerParams {
  const double* vel;       // [D][Nseg][3]
  const double* nhat;      // [Spad][3] sorted
  int n_det, n_seg, Spad, NG, group;
  double inv_q;
  int32_t* blk;            // [Spad/1024][Nseg][D][kBlockWords]
  unsigned* spread_max;    // float bits of max (hi - lo) of v.nhat/c over the groups
};

constexpr int kMaxSeriesTerms = 24;
constexpr int kMaxStageDet = 2;          // detectors the group kernel stages in shared memory
constexpr int kTileSegments = 32;

// dynamic shared memory of the group kernel for D detectors
size_t group_smem_bytes(int n_det);
// tile anchors of every (sorted template, tile) into anchors[Bpad * n_tiles * 2]
cudaError_t launch_anchors(const GroupParams& p, double* anchors, cudaStream_t st);

// launchers (return cudaError_t of the launch)
cudaError_t launch_doppler(const DopplerParams& p, cudaStream_t st);
cudaError_t launch_group(const GroupParams& p, bool half, bool record, bool weighted,
                         cudaStream_t st);
cudaError_t launch_lookup(const LookupParams& p, bool half, bool record, cudaStream_t st);
cudaError_t launch_topk(const float* psi, int Bpad, int B, int S, int k, const int32_t* bank_perm,
                        const int32_t* sky_perm, float* psi_out, int64_t* idx_out,
                        cudaStream_t st);
cudaError_t launch_unpermute(const float* src, int Spad, int Bpad, int S, int B,
                             const int32_t* sky_pos, const int32_t* bank_pos, float* dst,
                             cudaStream_t st);

// group-kernel geometry (shared by the host planner and the kernel)
constexpr int kGroupSkies = 16;     // skies per thread
constexpr int kGroupTmpl = 2;       // templates per thread
constexpr int kGroupUnits = 4;      // template pairs per work item
constexpr int kGroupWarps = 2;      // warps per unit
constexpr int kGroupLanes = 32 * kGroupWarps;             // sky groups per CTA
constexpr int kGroupTmplPerCta = kGroupUnits * kGroupTmpl;  // 8 templates per work item
constexpr int kSkyPad = kGroupSkies * kGroupLanes;        // 1024

}  // namespace tcw
