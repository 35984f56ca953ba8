// Internal declarations of libksconv (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ksconv.h"

namespace ksc {

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
int fit_split_lsq(const double *K, int lmax, int l_cut, double theta_cut,
                  const double *cl_in, int oversample, double rcond,
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
    float4 *d_tab;      // n_int intervals (output)
    double *d_nodes;    // 2*(n_int+1) scratch: node values, node slopes
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
    const float4 *d_tab;     // table
    int n_int;
    float inv_h;             // 1 / interval width
    float dc2;               // chord_cut^2
    double cos_cut;          // 1 - chord_cut^2 / 2
    float domega;            // 4 pi / Npix
};
cudaError_t launch_conv_general(const ConvPlan &p, const WorkItem *d_items,
                                int n_items, const float *d_in, float *d_out,
                                int n_maps, long long map_stride,
                                unsigned long long *d_count, cudaStream_t st);

// Largest table (intervals) a convolution kernel keeps in shared memory.
constexpr int kMaxIntervals = 8192;

} // namespace ksc

// The opaque split object.
struct ksc_split {
    int lmax = 0, l_cut = -1, nside = 0, mode = 0;
    int n_int = 0, n_unknowns = 0, n_kept = 0;
    double theta_cut = 0, chord_cut = 0, sigma_rms = 0, frac_error = 0;
    long long n_pairs = -1;
    std::vector<double> k_harm, c_real, k_tilde;

    // device state
    int device = 0;
    float4 *d_tab = nullptr;
    ksc::DevRing *d_rings = nullptr;
    int2 *d_range = nullptr;
    ksc::WorkItem *d_items = nullptr;
    int n_items = 0;
    std::vector<int> ring_first_item;  // nrings + 1 prefix offsets
    ksc::ConvPlan plan{};

    // end-to-end host path
    cudaStream_t own_stream = nullptr;
    float *d_io = nullptr;  // 2 * npix floats, allocated on first host call
};
