// K_r table build on the GPU (Sec. 3, Fig. 4: the real-space kernel that the
// convolution interpolates).
//
// Nodes sit at equal steps of the chord d = |r_i - r_j| = 2 sin(theta/2) on
// [0, d_cut]; z = cos(theta) = 1 - d^2/2.  For each node the kernel
//   K(z) = sum_{l<=lmax} (2l+1)/(4 pi) c_l P_l(z)
// and its slope dK/dd = -d K'(z) come from the FP64 three-term recurrence
// (one thread per node).  Each interval then stores the cubic Hermite
// polynomial through its two end nodes as FP32 coefficients in t = d/h - k:
//   K(t) = a0 + t (a1 + t (a2 + t a3)).
#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr double kInv4Pi = 0.07957747154594766788;  // 1 / (4 pi)

__global__ void node_values_kernel(const double *__restrict__ c, int lmax, int n_nodes,
                                   double h, double *__restrict__ nodeK,
                                   double *__restrict__ nodeD) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    const double d = h * (double)k;
    const double z = 1.0 - 0.5 * d * d;
    double p0 = 1.0, p1 = z;    // P_l, P_{l+1}
    double q0 = 0.0, q1 = 1.0;  // P'_l, P'_{l+1}
    double sk = c[0] * kInv4Pi, sd = 0.0;
    if (lmax >= 1) {
        sk += 3.0 * kInv4Pi * c[1] * z;
        sd += 3.0 * kInv4Pi * c[1];
    }
    for (int l = 1; l < lmax; ++l) {
        const double p2 = ((2.0 * l + 1.0) * z * p1 - (double)l * p0) / (double)(l + 1);
        const double q2 = q0 + (2.0 * l + 1.0) * p1;
        const double f = (2.0 * l + 3.0) * kInv4Pi * c[l + 1];
        sk = fma(f, p2, sk);
        sd = fma(f, q2, sd);
        p0 = p1; p1 = p2;
        q0 = q1; q1 = q2;
    }
    nodeK[k] = sk;
    nodeD[k] = -d * sd;  // dK/dd = dK/dz * dz/dd, dz/dd = -d
}

__global__ void hermite_coeff_kernel(const double *__restrict__ nodeK,
                                     const double *__restrict__ nodeD, int n_int, double h,
                                     int pad, float4 *__restrict__ tab) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (pad && k == n_int) {
        tab[k] = make_float4((float)nodeK[k], (float)(h * nodeD[k]), 0.0f, 0.0f);
        return;
    }
    if (k >= n_int) return;
    const double y0 = nodeK[k], y1 = nodeK[k + 1];
    const double m0 = h * nodeD[k], m1 = h * nodeD[k + 1];
    float4 c;
    c.x = (float)y0;
    c.y = (float)m0;
    c.z = (float)(3.0 * (y1 - y0) - 2.0 * m0 - m1);
    c.w = (float)(2.0 * (y0 - y1) + m0 + m1);
    tab[k] = c;
}

} // namespace

cudaError_t launch_table_build(const TableBuild &tb, cudaStream_t st) {
    const int n_nodes = tb.n_int + 1;
    double *nodeK = tb.d_nodes, *nodeD = tb.d_nodes + n_nodes;
    node_values_kernel<<<(n_nodes + 127) / 128, 128, 0, st>>>(tb.d_c, tb.lmax, n_nodes, tb.h,
                                                             nodeK, nodeD);
    hermite_coeff_kernel<<<(tb.n_int + 1 + 255) / 256, 256, 0, st>>>(nodeK, nodeD, tb.n_int,
                                                                   tb.h, tb.pad, tb.d_tab);
    return cudaGetLastError();
}

} // namespace ksc
