// Internal declarations of libksconv (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <nvtx3/nvToolsExt.h>
#include <string>
#include <vector>

#include "ksconv.h"

namespace ksc {

// NVTX range over a host-side scope (the enqueue of an asynchronous call, a split's
// construction): visible to a profiler's timeline, a no-op without one.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------------------
// HEALPix RING geometry (Gorski et al. 2005), rings r = 0 .. 4n-2 (ring number
// i = r + 1).  Pixel k of ring r sits at phi = (2k + phase) * pi / len.
// ---------------------------------------------------------------------------
struct RingGeom {
    std::vector<double> z, s;           // cos(theta), sin(theta), FP64
    std::vector<int> len, start, phase; // pixels, first pixel, phase flag (0/1)
};
void ring_geometry(int nside, RingGeom *g);

// Device copy of one ring (FP64 z and s feed the ring-pair constants).
struct DevRing {
    double z, s;
    int len, start, phase, pad;
};

// Geometry of one (output ring r, input ring q) pair, computed once per split
// on the host in FP64.  In table-position units (chord * n_int / chord_cut):
// u^2 = A + B sin^2(x), x = N * c with N the exact pixel-pair integer; hw is
// the half window in input pixels (dphi_max L_q / 2 pi + 1), negative when no
// pixel of q lies within theta_cut; w = ceil(dphi_max L_q / 2 pi) + 1 is the
// integer half window of the circulant belt kernel.
struct PairInfo {
    float Ah, Al, Bh, Bl, ch, cl;
    float hw;
    int w;
};

// Weight table of one ring pair for the symmetric gather.  For a fixed ring
// pair the kernel weight depends on the pixel pair only through the exact
// integer |N| (x = dphi / 2 = |N| c), so it is tabulated in |N|: cubic cells of
// 2^shift consecutive integers each, cell j covering j 2^shift <= |N| <
// (j + 1) 2^shift.  Because the width is a power of two, the cell of a pair and
// its offset in the cell, (|N| mod 2^shift) / 2^shift, are exact in FP32
// arithmetic (|N| < 2^24).  The width is the largest power of two that keeps a
// cell within kXRho intervals of the K_r table (in the chord) where the chord
// changes fastest, doubled (up to kXRhoMax intervals) while the cells would not
// fit a CTA's kXCap.  Pairs with |N| <= ncut lie within the cut.  ncell cells
// hold the cubic coefficients; the gather may read (without using) up to
// kXPad(L) cells beyond them, L the output ring's length.  ncell = 0: no table
// (whole-ring windows, or more cells than a CTA holds).
struct XInfo {
    int shift;  // cell width 2^shift in |N|
    int ncut;   // largest |N| within the cut
    int ncell;  // cells written (0: no table)
    int pad;
};
constexpr double kXRho = 2.0;     // chord-table intervals per cell (at most) ...
constexpr double kXRhoMax = 3.0;  // ... unless the cells would not fit
constexpr int kXCap = 4096;       // cells the largest gather tile holds (64 kB)
// Cells beyond ncell an edge quad of four positions may read: a quad reaches
// at most 3 positions (|N| steps of 2 L) past the cut.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline int kXPad(int L, int shift) { return ((6 * L) >> shift) + 2; }

// Weight table of one ring pair for the lockstep symmetric gather (conv_sym.cu).
// The eight lanes of a quarter warp walk the same input positions for classes
// C apart, so at one position their |N| differ by 2 lq C per lane (lq the input
// ring's length).  Cells of width 2 lq / m in |N| with m odd put those lanes m C
// cells apart: for odd C an odd step, so the eight 16-byte cells a quarter warp
// reads lie in eight different shared-memory bank groups.  A pair's table
// position is the rational P = (|N| m + off) / (2 lq): cell floor(P), offset
// P - floor(P), computed exactly from integers.  off puts a cell boundary
// between |N| = ncut (in the cut) and ncut + 1: cells 0 .. nct-1 hold cubics in
// the offset, cell nct is zero, and every position beyond it is clamped to it.
struct XOdd {
    int m;          // odd; cell width 2 lq / m
    int off;        // 0 <= off < 2 lq
    int nct;        // zero cell (0: no table)
    int ncut;       // largest |N| within the cut
    float cmh, cml; // c / m as a double-float pair: x of one unit of 2 lq j - off
    float hc;       // x extent of one cell, 2 lq c / m
    int pad;
};
constexpr double kXOddRho = 1.5;  // chord-table intervals per cell (at most) ...
// ... widened up to kXRhoMax while the cells would not fit (cells + 1 <= cap).
// The walk of a quarter warp visits positions up to (8 C) lq / L + 16 beyond a
// class's cut: the host keeps |N| there below 2^24 and |N| m + 2 lq below 2^31.
XOdd make_xodd(double A2, double B2, double c, double nint2, float hw, int L, int lq,
               double scale, int cap);

// Host: the table parameters of ring pair (r, q); A2, B2 are the ring-pair
// constants scaled to table-position units, c = pi / (2 L lq), L and lq the
// output and input rings' lengths, hw the window half-width (whole-ring windows
// get no table); scale <= 1 narrows the cells of a table coarser than the
// automatic size (n_int / n_auto).
XInfo make_xinfo(double A2, double B2, double c, double nint2, float hw, int L, int lq,
                 double scale);

// ---------------------------------------------------------------------------
// Host FP64 split fit (Sec. 2, Eq. 1-6).
// ---------------------------------------------------------------------------
struct FitResult {
    std::vector<double> k_harm;  // l = 0..l_cut
    std::vector<double> c_real;  // l = 0..lmax, Legendre coefficients of K_r
    std::vector<double> k_tilde; // l = 0..lmax, fitted kernel (Eq. 1)
    int n_unknowns = 0, n_kept = 0;
};
// Returns KSC_OK or an error code; *msg receives a reason on failure.
// n_constraints: 0 free real-space kernel, 1 K_r(theta_cut) = 0, 2 also
// dK_r/dz(theta_cut) = 0 (ksc_split_opts.cut_continuity).
int fit_split_lsq(const double *K, int lmax, int l_cut, double theta_cut,
                  const double *cl_in, int oversample, double rcond, int n_constraints,
                  FitResult *out, std::string *msg);

// Eq. 2 and Eq. 6 of a fitted kernel.
double sigma_rms_eq2(const double *K, const double *Kt, const double *cl, int lmax);
double frac_error_eq6(const double *K, const double *Kt, const double *cl,
                      int lmax, double alpha);

// ---------------------------------------------------------------------------
// Device launchers (csrc/*.cu).
// ---------------------------------------------------------------------------
struct TableBuild {
    const double *d_c;  // lmax+1 coefficients (device)
    int lmax;
    int n_int;
    double h;           // chord spacing
    float4 *d_tab;      // n_int intervals (output; n_int + 1 entries when pad is set)
    double *d_nodes;    // 2*(n_int+1) scratch: node values, node slopes
    int pad = 0;        // also write entry n_int: the constant-slope extension past d_cut,
                        // so that table position u = n_int needs no index clamp
};
cudaError_t launch_table_build(const TableBuild &tb, cudaStream_t st);

// Work item: a chunk of output pixels of one ring.
struct WorkItem {
    int ring;   // output ring (0-based)
    int k0;     // first output pixel within the ring
};

struct ConvPlan {
    int nside, npix, nrings;
    const DevRing *d_rings;  // nrings
    const int2 *d_range;     // per output ring: first/last input ring (0-based)
    const PairInfo *d_pairs; // ring-pair geometry, d_pair_base[r] + (q - range.x)
    const XInfo *d_xinfo;    // x tables of the symmetric gather, same indexing
    const XOdd *d_xodd;      // odd-step tables of the lockstep gather, same indexing
    const int *d_pair_base;
    const float4 *d_tab;     // table
    int n_int;
    float inv_h;             // 1 / interval width
    float dc2;               // chord_cut^2
    double cos_cut;          // 1 - chord_cut^2 / 2
    float domega;            // 4 pi / Npix
    int belt_lo, belt_hi;    // 0-based ring indices of the equatorial belt
    double scale2;           // (n_int / chord_cut)^2: chord^2 -> table position^2
    float belt_c1h, belt_c1l; // pi / (2 L_belt) as a double-float pair
    float nint2;             // the cut in table-position^2 units (n_int^2)
};
// General ring-pair gather.  With belt_split set, belt output rings only take
// their polar-cap input rings and add them to the output (the belt kernel has
// written the belt-belt part); cap output rings take every input ring.
// Counting (d_count != NULL): belt_split 0 counts every in-disc pair, 1 only
// belt-belt pairs, 2 every other pair.
cudaError_t launch_conv_general(const ConvPlan &p, const WorkItem *d_items,
                                int n_items, const float *d_in, float *d_out,
                                int n_maps, long long map_stride, int belt_split,
                                unsigned long long *d_count, cudaStream_t st);

// Circulant belt-belt kernel; items are (belt ring, first pixel) chunks of
// belt_chunk() pixels; seg_cap floats per shared-memory buffer.
int belt_chunk();
cudaError_t launch_conv_belt(const ConvPlan &p, const int2 *d_items, int n_items,
                             int seg_cap, const float *d_in, float *d_out, int n_maps,
                             long long map_stride, int *d_err, cudaStream_t st);

// tcgen05 multi-map kernel for belt ring pairs: items are (belt ring, first
// pixel) blocks of belt_mma_block() outputs; maps in groups of belt_mma_maps().
int belt_mma_block();
int belt_mma_maps();
size_t belt_mma_smem(int w_cap);
size_t belt_mma_workspace_floats(int n_belt, int n_tiles, int n_maps);
cudaError_t launch_conv_belt_mma(const ConvPlan &p, const int2 *d_items, int n_items, int w_cap,
                                 int n_tiles, int ext0, float *d_ws, const float *d_in,
                                 float *d_out, int n_maps, long long map_stride, int *d_err,
                                 cudaStream_t st);

// Symmetric gather over northern rings (and the equator): each thread owns
// one first-quarter position and writes its eight images; only output rings
// in [band_lo, band_hi] are written.  Items are (ring, first quarter position)
// chunks of sym_chunk(nside) classes (the tile launch_conv_sym uses for that nside).
int sym_chunk(int nside);
int sym_classes(int len, int phase);  // reflection classes of a ring's first quarter
// CTAs claim items in list order through per-call counters taken from the
// stream-ordered allocator.
cudaError_t launch_conv_sym(const ConvPlan &p, const WorkItem *d_items, int n_items,
                            const float *d_in, float *d_out, int n_maps,
                            long long map_stride, int belt_split, int band_lo,
                            int band_hi, int *d_err, cudaStream_t st);

// ---------------------------------------------------------------------------
// Batched persistent launches (csrc/batch.cpp).  An entry is one map convolved
// with one split; items are int4 {entry, ring, first pixel or class, 0}.
// The tile variant selects a kernel's block shape (the autotuned tile): belt
// variant 0 / 1 = full / half block (belt_variant_chunk(v) outputs per item);
// gather variant 0 / 1 = full / half block, 2 = paired lanes
// (sym_variant_chunk(v) reflection classes per item).  CTAs claim items from *d_counter,
// which must be zero at launch.  per_sm_cap > 0 caps the resident CTAs per SM.
// ---------------------------------------------------------------------------
struct BatchEntry {
    const float *in;
    float *out;
    int plan;        // index into the batch's ConvPlan array
    int belt_split;  // 1: the belt kernel wrote this entry's belt-belt part
};
int belt_variant_chunk(int variant);  // variants 0, 1
int sym_variants();                   // number of gather variants
int sym_variant_chunk(int variant);
cudaError_t launch_conv_belt_batch(int variant, const ConvPlan *d_plans,
                                   const BatchEntry *d_entries, const int4 *d_items, int n_items,
                                   int seg_cap, int per_sm_cap, int *d_err, int *d_counter,
                                   cudaStream_t st);
cudaError_t launch_conv_sym_batch(int variant, const ConvPlan *d_plans,
                                  const BatchEntry *d_entries, const int4 *d_items, int n_items,
                                  int per_sm_cap, int *d_counter, int *d_err, cudaStream_t st);

// tcgen05 gather for map stacks (symmetric ring pairs): items are the
// symmetric work items of sym_mma_chunk() classes each; maps in groups of
// sym_mma_maps(); same outputs as launch_conv_sym over the whole map.
int sym_mma_maps();
int sym_mma_chunk();

// tcgen05 gather for single maps (grid.y over maps of a stack): items of
// sym_tc_chunk() classes (the same items as the map-stack kernel); same outputs
// as launch_conv_sym, written for output rings in [band_lo, band_hi].
int sym_tc_chunk();
cudaError_t launch_conv_sym_tc(const ConvPlan &p, const WorkItem *d_items, int n_items,
                               const float *d_in, float *d_out, int n_maps, long long map_stride,
                               int belt_split, int band_lo, int band_hi, int *d_err,
                               cudaStream_t st);
cudaError_t launch_conv_sym_mma(const ConvPlan &p, const WorkItem *d_items, int n_items,
                                const float *d_in, float *d_out, int n_maps,
                                long long map_stride, int belt_split, int *d_err,
                                cudaStream_t st);

// Record the message returned by ksc_last_error() on this thread.
void set_last_error(const std::string &msg);

// Host-side fault injection for tests (no GPU fault is ever made): the
// environment variable KSC_FAULT = "alloc:N" makes the N-th device allocation of
// each split construction or host-path call fail as if the device were out of
// memory (N >= 1).  Returns true when allocation number `n` (1-based) must fail.
bool inject_alloc_fault(int n);
// GPU spherical-harmonic transforms (sht.cu): synthesis (add != 0 adds to the
// map) and analysis (each a_lm scaled by d_kl[l] when d_kl is given); alm are
// complex doubles in m-major order, sht_n_alm(lmax) of them.
cudaError_t sht_synthesis(int nside, int lmax, const double2 *d_alm, float *d_map, int add,
                          cudaStream_t st);
cudaError_t sht_analysis(int nside, int lmax, const float *d_map, const double *d_kl,
                         double2 *d_alm, cudaStream_t st);
long long sht_n_alm(int lmax);

// Largest table (intervals) a convolution kernel keeps in shared memory.
constexpr int kMaxIntervals = 8192;

} // namespace ksc

// The opaque split object.
struct ksc_split {
    int lmax = 0, l_cut = -1, nside = 0, mode = 0;
    int n_int = 0, n_unknowns = 0, n_kept = 0;
    double theta_cut = 0, chord_cut = 0, sigma_rms = 0, frac_error = 0;
    long long n_pairs = -1, n_pairs_belt = -1;
    std::vector<double> k_harm, c_real, k_tilde;

    // device state
    int device = 0;
    float4 *d_tab = nullptr;
    ksc::DevRing *d_rings = nullptr;
    int2 *d_range = nullptr;
    ksc::PairInfo *d_pairs = nullptr;
    ksc::XInfo *d_xinfo = nullptr;
    ksc::XOdd *d_xodd = nullptr;
    double frac_tabulated = 0.0;  // share of gather weights from dphi tables
    int *d_pair_base = nullptr;
    // work lists, each with a per-ring prefix (nrings + 1 offsets)
    ksc::WorkItem *d_items = nullptr;   // every ring (pair counting)
    int n_items = 0;
    std::vector<int> ring_first_item;
    ksc::WorkItem *d_items_sym = nullptr;  // northern rings for the symmetric gather
    ksc::WorkItem *d_items_sym_lpt = nullptr;  // the same items, longest first (whole map)
    int n_items_sym = 0;
    ksc::WorkItem *d_items_smma = nullptr;  // 128-class items of the tensor cap kernels,
    ksc::WorkItem *d_items_smma_lpt = nullptr;  // in ring order and longest first
    int n_items_smma = 0;
    std::vector<int> ring_first_smma;
    int cap_kernel = 0;                    // ksc_split_opts.cap_kernel
    std::vector<int> ring_first_sym;
    int path = 0;                          // 0: belt + symmetric, 1: general only
    int2 *d_items_belt = nullptr;          // belt chunks for the circulant kernel
    int n_items_belt = 0;
    std::vector<int> ring_first_belt;
    int seg_cap = 0;
    int max_nd = 0;                        // widest circulant weight window (belt pairs)
    std::vector<double> cost_belt, cost_sym; // per ring: window positions per output pixel
    int2 *d_items_mma = nullptr;           // 128-output belt blocks for the tensor kernel
    int n_items_mma = 0;
    int w_cap = 0;                         // widest belt weight window
    int tensor = 0;                        // ksc_split_opts.tensor (0, 1, 2)
    int mma_ext0 = 0, mma_ntiles = 0;      // ring extension and K tiles per belt ring
    float *d_ws = nullptr;                 // pre-tiled map stack (tensor path workspace)
    size_t ws_floats = 0;
    int *d_err = nullptr;                  // device error flag (bounded waits)
    ksc::ConvPlan plan{};

    // end-to-end host path (one call at a time per split: host_mu)
    std::mutex host_mu;
    cudaStream_t own_stream = nullptr;
    float *d_io = nullptr;  // 2 * npix floats, allocated on first host call
};
