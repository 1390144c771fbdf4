// Device code of the fluctuating D3Q19 LB + bead-spring chain step.
//
// Storage: populations in structure-of-arrays planes pop[i][z][y][x] (plane stride
// `plane` elements), two buffers A/B.  FP32/BF16/FP16 contexts store the deviation
// n_i - w_i rho0 (DEV = true), the FP64 context the full n_i.  A step reads buffer A
// (post-collision populations of the previous step, "pull" storage) and writes B.
//
// One step = k_bead_step (one thread block, or a cluster of up to 8: velocity Verlet,
// FENE/WCA, interpolation, friction + noise, spreading -> sparse list of per-node population
// corrections), k_lb_step (every node: pull-stream, moments, relaxation + noise,
// back-transform) and the force corrections, added to B by k_apply_pending or, kept pending,
// by the next step's kernels where they read.  The bead kernel and the LB kernel read only A,
// so they are independent; the correction is additive on the post-collision populations
// because the collision conserves the density and momentum it depends on.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "d3q19.cuh"
#include "philox.cuh"

namespace gblb {

enum : unsigned { ST_FENE = 1u, ST_NONFINITE = 2u, ST_TIMEOUT = 4u };

// ---------------------------------------------------------------------------------------
// storage <-> arithmetic conversions
// ---------------------------------------------------------------------------------------
template <class S, class R>
__device__ __forceinline__ R ld(const S* p) { return (R)(*p); }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16, float>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ float ld<__half, float>(const __half* p) { return __half2float(*p); }

template <class S, class R>
__device__ __forceinline__ void st(S* p, R v) { *p = (S)v; }
template <>
__device__ __forceinline__ void st<__nv_bfloat16, float>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ void st<__half, float>(__half* p, float v) { *p = __float2half_rn(v); }

// two consecutive elements (the first at an even element offset, so 2 sizeof(S)-aligned) in
// one access: 8 bytes for FP32, 16 for FP64, 4 for the 16-bit formats
template <class S, class R>
__device__ __forceinline__ void ld2(const S* p, R& a, R& b);
template <>
__device__ __forceinline__ void ld2<float, float>(const float* p, float& a, float& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = v.x;
  b = v.y;
}
template <>
__device__ __forceinline__ void ld2<double, double>(const double* p, double& a, double& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = v.x;
  b = v.y;
}
template <>
__device__ __forceinline__ void ld2<__nv_bfloat16, float>(const __nv_bfloat16* p, float& a, float& b) {
  const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
  a = __low2float(v);
  b = __high2float(v);
}
template <>
__device__ __forceinline__ void ld2<__half, float>(const __half* p, float& a, float& b) {
  const __half2 v = *reinterpret_cast<const __half2*>(p);
  a = __low2float(v);
  b = __high2float(v);
}
template <class S, class R>
__device__ __forceinline__ void st2(S* p, R a, R b);
template <>
__device__ __forceinline__ void st2<float, float>(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
template <>
__device__ __forceinline__ void st2<double, double>(double* p, double a, double b) {
  *reinterpret_cast<double2*>(p) = make_double2(a, b);
}
template <>
__device__ __forceinline__ void st2<__nv_bfloat16, float>(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}
template <>
__device__ __forceinline__ void st2<__half, float>(__half* p, float a, float b) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}

// 1/rho for the LB kernel: the hardware reciprocal in single precision (1 ulp; the density is
// a normal number), correctly rounded division in double
template <class R>
__device__ __forceinline__ R lb_rcp(R x) { return R(1) / x; }
template <>
__device__ __forceinline__ float lb_rcp<float>(float x) { return approx_rcp(x); }

// ---------------------------------------------------------------------------------------
// kernel parameter blocks (passed by value)
// ---------------------------------------------------------------------------------------
template <class R>
struct FluidK {
  unsigned L;
  unsigned long long plane;  // elements between population planes
  R rho0;
  R gs, gb;        // relaxation eigenvalues: shear modes 5..9, bulk mode 4 (kinetic modes: 0)
  R cnoise[Q];     // sqrt(mu b_k (1 - gamma_k^2)), mode k's noise per sqrt(rho); 0 if silent
  // the same relaxation and noise in terms of the scaled moments a_k = m*_k / b_k used by the
  // back-transform: a_k = am_k m_k + ae_k m_eq,k + ag_k sqrt(rho) g_k  (k = 4..18)
  R am[Q], ae[Q], ag[Q];
  // the same times w_2 = 1/36, the weight of the next-nearest velocities, which the forward
  // kernel's back-transform then needs no more multiplications for
  R wam[Q], wae[Q], wag[Q];
  uint32_t k0, k1; // Philox key of the fluid stream
  RoundKeys rk;    // its ten round keys
  int ncalls;      // Philox calls per node: 0 (noise off), 1 (stress modes only), 2 (all)
  int body_on;     // uniform body force
  R body_dJ[3];    // lattice momentum it adds per step and node: f h^2 / a
  unsigned long long* nonpos;  // counter of non-positive densities met by the noise
  int pdl;         // launch chaining of the LB kernel: bit 0 waits for the previous grid before
                   // reading, bit 1 waits for it before completing (see k_lb_step)
  int angle_tab;   // double precision: the LB kernel's Box-Muller angles from per-block tables
  // null, or a device counter the step kernels add their step argument to (graph replays of a
  // fixed sequence of launches at other step numbers)
  const uint32_t* d_step;
};

// the step number of a launch: its argument, offset by the device counter when there is one
template <class R>
__device__ __forceinline__ uint32_t launch_step(const FluidK<R>& P, uint32_t step) {
  return P.d_step ? *P.d_step + step : step;
}

// *p = v on the stream (a device step counter before a graph replay)
template <class T>
__global__ void k_store_value(T* p, T v) { *p = v; }

template <class R>
struct ChainK {
  int N;
  R m, zeta, kfene, R0sq, eps, sig2, rc2;
  R h, a, box, half_box;
  R amp;            // sqrt(2 kT zeta / h), 0 without bead noise
  uint32_t k0, k1;  // Philox key of the bead stream
  R ext[3];         // constant external force on each bead
  R u_scale;        // a / h (h: the LB step): lattice -> physical velocity
  R inv_a3;         // 1 / a^3
  R dJ_scale;       // h^2 / a: force density -> lattice momentum per LB step
  int nsub;         // MD steps per LB step (h above is the MD step h_LB / nsub)
  R spread;         // 1 / nsub: each MD step's reaction, averaged over the LB step
  R* fc_hist;       // nsub x 3N coupling forces of the MD substeps
  // bead state (global, 3N each, bead-major).  The bead kernel reads the state at the start
  // of a step from the *_in arrays (normally the same arrays; the adjoint's recomputation
  // reads one saved state and writes the next) and writes the end state to x .. Fc
  const R *x_in, *xl_in, *v_in, *F_in;
  const int* img_in;
  R* x;    // wrapped positions in [0, box): high part
  R* xl;   // low part: position = x + xl + img * box (compensated, ~2x the precision of R)
  int* img;  // periodic image counters
  R* v;
  R* F;    // total force of the last step (F_cons + F_c)
  R* Fc;   // coupling force of the last step
  // scratch (global)
  R* vh;       // 3N half-step velocities
  R* fcons;    // 3N conservative forces
  int* e_node;  // 8N corner nodes
  R* e_w;      // 8N trilinear weights
  R* e_mom;    // 4 x 8N: post-stream rho, Jx, Jy, Jz at the corner node
  int4* p_pos; // pending force corrections: {node, x, y, z}, and 19 deltas [i][cap]
  R* p_dn;
  int* p_count;
  int cap;     // 8N
  unsigned* status;
  // FP64 snapshot of the state after each step, written by the bead kernel of step k into
  // slot k mod 2 (3N unwrapped positions x + xl + img box, then 3N velocities), or null
  double* snap;
  double snap_box;  // L a in FP64
};

// Force corrections in flight between consecutive steps of a multi-step run.  The bead kernel
// of step k writes them twice: as a list (node, 19 deltas) for the final flush, and into a
// dense correction field of the population layout [i][plane] that is zero except at pending
// nodes; it also marks, in a bit mask over the nodes (one 32-bit word per 32 consecutive
// linear indices), every node that pulls from a corrected node.  The LB kernel of step k+1
// adds the dense field to what it pulls at marked nodes, and the bead kernel of step k+1 to
// what it gathers.  Two slots alternate by step; a bead kernel first clears its slot's dense
// entries and mask words of the list from two steps before, and a flush clears what it
// applies.
template <class R>
struct PendK {
  int have_prev;          // 0: nothing pending (the stored populations are complete)
  const unsigned* prev_mask;  // nodes that pull from the previous step's corrected nodes
  const R* prev_dense;    // the previous step's corrections, dense
  int4* cur_pos;          // this step's list: {node, x, y, z}
  R* cur_dn;              // 19 deltas [i][cap]
  int* cur_count;
  R* cur_dense;           // this step's slot of the dense field
  unsigned* cur_mask;     // this step's slot of the mask (cleared of the old list)
  int mark;               // 1: mark the pulling nodes of this step's list (deferred steps)
  int cap;
  unsigned long long plane;  // element stride between the 19 planes
  unsigned seg0;             // index of this box's first word in the mask arrays
};

constexpr int kSegShift = 5;  // mask words of 32 consecutive nodes

// ---------------------------------------------------------------------------------------
// moment algebra
// ---------------------------------------------------------------------------------------
// scaled moments a_k = m_k / b_k  ->  populations n_i = w_i sum_k e_k(c_i) a_k
template <class R>
__device__ __forceinline__ void modes_to_pops(const R a[Q], R out[Q]) {
  {
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int c = basis(k, 0);
      if (c != 0) acc += R(c) * a[k];
    }
    out[0] = acc * (R(w36(0)) / R(36));
  }
#pragma unroll
  for (int p = 0; p < NPAIR; ++p) {
    const int i = 2 * p + 1;
    R S = R(0), D = R(0);
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const int c = basis(k, i);
      if (c == 0) continue;
      if (odd_mode(k))
        D += R(c) * a[k];
      else
        S += R(c) * a[k];
    }
    const R w = R(w36(i)) / R(36);
    out[i] = w * (S + D);
    out[i + 1] = w * (S - D);
  }
}

template <int K>
struct InvB {
  static constexpr double v = 36.0 / (double)norm36(K);
};

// Moment increments (modes 1..9) of a force adding lattice momentum dJ at a node of
// density rho and pre-collision momentum J (second-order forcing reading):
//   dm_1..3 = dJ;  dPi = (1+g_s)/2 (U'dJ + dJU' - 2/3 1 U'.dJ) + (1+g_b)/3 1 U'.dJ,
//   U' = (J + dJ/2)/rho, mapped onto modes 4..9.
template <class R>
__device__ __forceinline__ void force_moments(R rho, R jx, R jy, R jz, R dx, R dy, R dz, R gs,
                                              R gb, R dm[10]) {
  const R ir = R(1) / rho;
  const R ux = (jx + R(0.5) * dx) * ir, uy = (jy + R(0.5) * dy) * ir, uz = (jz + R(0.5) * dz) * ir;
  const R ud = ux * dx + uy * dy + uz * dz;
  const R cs = R(0.5) * (R(1) + gs);
  const R diag = ((R(1) + gb) / R(3) - R(2) / R(3) * cs) * ud;
  const R pxx = R(2) * cs * ux * dx + diag;
  const R pyy = R(2) * cs * uy * dy + diag;
  const R pzz = R(2) * cs * uz * dz + diag;
  dm[0] = R(0);
  dm[1] = dx;
  dm[2] = dy;
  dm[3] = dz;
  dm[4] = pxx + pyy + pzz;
  dm[5] = R(2) * pxx - pyy - pzz;
  dm[6] = pyy - pzz;
  dm[7] = cs * (ux * dy + uy * dx);
  dm[8] = cs * (uy * dz + uz * dy);
  dm[9] = cs * (ux * dz + uz * dx);
}

// population deltas of moment increments dm_0..9
template <class R>
__device__ __forceinline__ void dmoments_to_dpops(const R dm[10], R out[Q]) {
  R a[Q];
  a[0] = dm[0];
  a[1] = dm[1] * R(InvB<1>::v);
  a[2] = dm[2] * R(InvB<2>::v);
  a[3] = dm[3] * R(InvB<3>::v);
  a[4] = dm[4] * R(InvB<4>::v);
  a[5] = dm[5] * R(InvB<5>::v);
  a[6] = dm[6] * R(InvB<6>::v);
  a[7] = dm[7] * R(InvB<7>::v);
  a[8] = dm[8] * R(InvB<8>::v);
  a[9] = dm[9] * R(InvB<9>::v);
#pragma unroll
  for (int k = 10; k < Q; ++k) a[k] = R(0);
  modes_to_pops(a, out);
}

// ---------------------------------------------------------------------------------------
// explicit D3Q19 transforms in the ABI velocity order (pairs 2p+1, 2p+2 opposite):
// the same linear maps as the basis tables above, with the sums shared between modes and
// between populations written out, which the compiler cannot do itself without reassociating
// floating-point sums.
// ---------------------------------------------------------------------------------------
// moments 0..9 (density, momentum, stress modes) of 19 populations
template <class R>
__host__ __device__ __forceinline__ void moments_0_9(const R n[Q], R m[10]) {
  const R s0 = n[1] + n[2], d0 = n[1] - n[2];
  const R s1 = n[3] + n[4], d1 = n[3] - n[4];
  const R s2 = n[5] + n[6], d2 = n[5] - n[6];
  const R s3 = n[7] + n[8], d3 = n[7] - n[8];
  const R s4 = n[9] + n[10], d4 = n[9] - n[10];
  const R s5 = n[11] + n[12], d5 = n[11] - n[12];
  const R s6 = n[13] + n[14], d6 = n[13] - n[14];
  const R s7 = n[15] + n[16], d7 = n[15] - n[16];
  const R s8 = n[17] + n[18], d8 = n[17] - n[18];
  const R sxy = s3 + s4, sxz = s5 + s6, syz = s7 + s8;
  const R snn = sxy + sxz + syz;
  m[0] = n[0] + (s0 + s1 + s2) + snn;
  m[1] = d0 + d3 + d4 + d5 + d6;
  m[2] = d1 + d3 - d4 + d7 + d8;
  m[3] = d2 + d5 - d6 + d7 - d8;
  m[4] = snn - n[0];
  m[5] = R(2) * (s0 - syz) - s1 - s2 + sxy + sxz;
  m[6] = s1 - s2 + sxy - sxz;
  m[7] = s3 - s4;
  m[8] = s7 - s8;
  m[9] = s5 - s6;
}

// populations n_i = w_i sum_k e_k(c_i) a_k from scaled moments a_k = m_k / b_k
template <class R>
__host__ __device__ __forceinline__ void pops_from_scaled(const R a[Q], R n[Q]) {
  const R w0 = R(1) / R(3), w1 = R(1) / R(18), w2 = R(1) / R(36);
  n[0] = w0 * (a[0] - a[4] + a[16]);
  // nearest neighbours
  const R t = a[0] - a[5] - R(2) * a[16] + a[17];
  const R Sx = a[0] + R(2) * (a[5] - a[16] - a[17]);
  const R Sy = t + (a[6] - a[18]);
  const R Sz = t - (a[6] - a[18]);
  const R Dx = a[1] - R(2) * a[10], Dy = a[2] - R(2) * a[11], Dz = a[3] - R(2) * a[12];
  n[1] = w1 * (Sx + Dx);
  n[2] = w1 * (Sx - Dx);
  n[3] = w1 * (Sy + Dy);
  n[4] = w1 * (Sy - Dy);
  n[5] = w1 * (Sz + Dz);
  n[6] = w1 * (Sz - Dz);
  // next-nearest neighbours
  const R base = a[0] + a[4] + a[16];
  const R P = a[5] + a[17], Qv = a[6] + a[18];
  const R X = base + P + Qv, Y = base + P - Qv, Z = base - R(2) * P;
  const R A = a[1] + a[10], B = a[2] + a[11], Cc = a[3] + a[12];
  const R D3 = (A + B) + (a[13] - a[14]);
  const R D4 = (A - B) + (a[13] + a[14]);
  const R D5 = (A + Cc) - (a[13] - a[15]);
  const R D6 = (A - Cc) - (a[13] + a[15]);
  const R D7 = (B + Cc) + (a[14] - a[15]);
  const R D8 = (B - Cc) + (a[14] + a[15]);
  const R S3 = X + a[7], S4 = X - a[7];
  const R S5 = Y + a[9], S6 = Y - a[9];
  const R S7 = Z + a[8], S8 = Z - a[8];
  n[7] = w2 * (S3 + D3);
  n[8] = w2 * (S3 - D3);
  n[9] = w2 * (S4 + D4);
  n[10] = w2 * (S4 - D4);
  n[11] = w2 * (S5 + D5);
  n[12] = w2 * (S5 - D5);
  n[13] = w2 * (S6 + D6);
  n[14] = w2 * (S6 - D6);
  n[15] = w2 * (S7 + D7);
  n[16] = w2 * (S7 - D7);
  n[17] = w2 * (S8 + D8);
  n[18] = w2 * (S8 - D8);
}

// the same map from w_2-scaled moments a'_k = a_k / 36: n_0 = 12 (...), nearest-neighbour
// populations 2 (S' +- D'), next-nearest S' +- D'
template <class R>
__host__ __device__ __forceinline__ void pops_from_w2scaled(const R a[Q], R n[Q]) {
  n[0] = R(12) * (a[0] - a[4] + a[16]);
  const R t = a[0] - a[5] - R(2) * a[16] + a[17];
  const R Sx = a[0] + R(2) * (a[5] - a[16] - a[17]);
  const R Sy = t + (a[6] - a[18]);
  const R Sz = t - (a[6] - a[18]);
  const R Dx = a[1] - R(2) * a[10], Dy = a[2] - R(2) * a[11], Dz = a[3] - R(2) * a[12];
  n[1] = R(2) * (Sx + Dx);
  n[2] = R(2) * (Sx - Dx);
  n[3] = R(2) * (Sy + Dy);
  n[4] = R(2) * (Sy - Dy);
  n[5] = R(2) * (Sz + Dz);
  n[6] = R(2) * (Sz - Dz);
  const R base = a[0] + a[4] + a[16];
  const R P = a[5] + a[17], Qv = a[6] + a[18];
  const R X = base + P + Qv, Y = base + P - Qv, Z = base - R(2) * P;
  const R A = a[1] + a[10], B = a[2] + a[11], Cc = a[3] + a[12];
  const R D3 = (A + B) + (a[13] - a[14]);
  const R D4 = (A - B) + (a[13] + a[14]);
  const R D5 = (A + Cc) - (a[13] - a[15]);
  const R D6 = (A - Cc) - (a[13] + a[15]);
  const R D7 = (B + Cc) + (a[14] - a[15]);
  const R D8 = (B - Cc) + (a[14] + a[15]);
  const R S3 = X + a[7], S4 = X - a[7];
  const R S5 = Y + a[9], S6 = Y - a[9];
  const R S7 = Z + a[8], S8 = Z - a[8];
  n[7] = S3 + D3;
  n[8] = S3 - D3;
  n[9] = S4 + D4;
  n[10] = S4 - D4;
  n[11] = S5 + D5;
  n[12] = S5 - D5;
  n[13] = S6 + D6;
  n[14] = S6 - D6;
  n[15] = S7 + D7;
  n[16] = S7 - D7;
  n[17] = S8 + D8;
  n[18] = S8 - D8;
}

// ---------------------------------------------------------------------------------------
// LB kernel: pull-stream + collide for every node (Sec. II B, Eq. 3)
// ---------------------------------------------------------------------------------------
// Collide the 19 pulled populations n of one node (Sec. II B, Eq. 3) into its 19
// post-collision populations out (lb_collide_store: written to dst at element offset
// i * pl + node for population i).
template <class R, bool DEV, bool NOISE>
__device__ __forceinline__ void lb_collide(const R* n, R out[Q], const FluidK<R>& P, const RoundKeys& rk,
                                           unsigned long long* nonpos, const uint32_t step, const unsigned node,
                                           const AngleTab* tab = nullptr) {
  // moments 0..9 (the kinetic modes relax to zero and are not needed)
  R m[10];
  moments_0_9<R>(n, m);
  const R rho = DEV ? P.rho0 + m[0] : m[0];
  const R jx = m[1], jy = m[2], jz = m[3];
  const R ir = lb_rcp<R>(rho);
  const R xx = jx * jx * ir, yy = jy * jy * ir, zz = jz * jz * ir;
  // post-collision moments, directly as w_2-scaled moments a'_k = m*_k / (36 b_k): relaxation
  // of the stress modes towards equilibrium (Eq. 4), kinetic modes to zero, plus the
  // fluctuating part sqrt(rho) phi_k g_k / (36 b_k)
  R a[Q];
  a[0] = m[0] * R(1.0 / 36.0);
  a[1] = jx * R(InvB<1>::v / 36.0);
  a[2] = jy * R(InvB<2>::v / 36.0);
  a[3] = jz * R(InvB<3>::v / 36.0);
  {
    const R e4 = xx + yy + zz, e5 = R(2) * xx - yy - zz, e6 = yy - zz;
    const R e7 = jx * jy * ir, e8 = jy * jz * ir, e9 = jx * jz * ir;
    a[4] = P.wam[4] * m[4] + P.wae[4] * e4;
    a[5] = P.wam[5] * m[5] + P.wae[5] * e5;
    a[6] = P.wam[6] * m[6] + P.wae[6] * e6;
    a[7] = P.wam[7] * m[7] + P.wae[7] * e7;
    a[8] = P.wam[8] * m[8] + P.wae[8] * e8;
    a[9] = P.wam[9] * m[9] + P.wae[9] * e9;
  }
#pragma unroll
  for (int k = 10; k < Q; ++k) a[k] = R(0);

  if (NOISE) {
    if (!(rho > R(0))) atomicAdd(nonpos, 1ull);
    fluid_noise<R>(step, node, rk, P.ncalls > 1, NoiseScale<R>(rho),
                   [&](int j, R g) { a[4 + j] += P.wag[4 + j] * g; }, tab);
  }

  if (P.body_on) {
    R dm[10];
    force_moments(rho, jx, jy, jz, P.body_dJ[0], P.body_dJ[1], P.body_dJ[2], P.gs, P.gb, dm);
    a[1] += dm[1] * R(InvB<1>::v / 36.0);
    a[2] += dm[2] * R(InvB<2>::v / 36.0);
    a[3] += dm[3] * R(InvB<3>::v / 36.0);
    a[4] += dm[4] * R(InvB<4>::v / 36.0);
    a[5] += dm[5] * R(InvB<5>::v / 36.0);
    a[6] += dm[6] * R(InvB<6>::v / 36.0);
    a[7] += dm[7] * R(InvB<7>::v / 36.0);
    a[8] += dm[8] * R(InvB<8>::v / 36.0);
    a[9] += dm[9] * R(InvB<9>::v / 36.0);
  }

  pops_from_w2scaled<R>(a, out);
}

// The two nodes of a thread as the two lanes of packed single-precision arithmetic
// (add.f32x2, mul.f32x2, fma.f32x2: one instruction for both nodes, each lane rounded as the
// scalar operation), so that the moment transforms above serve both nodes at once.
struct f2 {
  float2 v;
  __device__ __forceinline__ f2() {}
  __device__ __forceinline__ explicit f2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ f2 mk2(float2 v) {
  f2 r;
  r.v = v;
  return r;
}
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return mk2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return mk2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return mk2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return mk2(__ffma2_rn(a.v, b.v, c.v)); }

// Box-Muller pairs of the noise words w0 (node) and w1 (node + 1): lane by lane the
// arithmetic of fluid_pair<float>, the special-function operations per lane, the rest packed.
template <bool SECOND>
__device__ __forceinline__ void fluid_pair2(uint32_t w0, uint32_t w1, f2 cl, f2& g, f2& h) {
  const f2 u0 = f2(fluid_radius_1p(w0), fluid_radius_1p(w1)) - f2(0x1.fffff8p-1f);  // (k_r + 1/2) 2^-21
  const f2 t = f2(1.0f) - u0;
  const f2 ser = t * fma2(t, fma2(t, f2(-0.480898347f), f2(-0.721347520f)), f2(-1.44269504f));
  const f2 l2(t.v.x < 1.0e-3f ? ser.v.x : approx_lg2(u0.v.x), t.v.y < 1.0e-3f ? ser.v.y : approx_lg2(u0.v.y));
  const f2 x = cl * l2;
  const f2 r = x * f2(approx_rsqrt(x.v.x), approx_rsqrt(x.v.y));
  const f2 d = f2(fluid_angle_1p(w0), fluid_angle_1p(w1)) - f2(1.5f);  // k_a 2^-11 - 1/2, exact
  const f2 th = fma2(f2(6.28318530717958647692f), d, f2(1.53398078788564123e-3f));
  g = r * f2(approx_cos(th.v.x), approx_cos(th.v.y));
  if (SECOND) h = r * f2(approx_sin(th.v.x), approx_sin(th.v.y));
}
template <int PR, bool SECOND = true, class Emit>
__device__ __forceinline__ void fluid_pair2_emit(uint32_t w0, uint32_t w1, f2 cl, Emit& emit) {
  f2 g, h;
  fluid_pair2<SECOND>(w0, w1, cl, g, h);
  emit(2 * PR, g);
  if (SECOND) emit(2 * PR + 1, h);
}
// fluid_noise for the nodes (node, node + 1) at once: emit(j, (g_j of node, g_j of node + 1))
template <class Emit>
__device__ __forceinline__ void fluid_noise2(uint32_t step, uint32_t node, const RoundKeys& rk, bool kinetic, f2 cl,
                                             Emit emit) {
  U4 a = philox4x32_10_rk(U4{step, node, 0u, 0u}, rk);
  U4 b = philox4x32_10_rk(U4{step, node + 1u, 0u, 0u}, rk);
  fluid_pair2_emit<0>(a.x, b.x, cl, emit);
  fluid_pair2_emit<1>(a.y, b.y, cl, emit);
  fluid_pair2_emit<2>(a.z, b.z, cl, emit);
  if (!kinetic) return;
  fluid_pair2_emit<3>(a.w, b.w, cl, emit);
  a = philox4x32_10_rk(U4{step, node, 1u, 0u}, rk);
  b = philox4x32_10_rk(U4{step, node + 1u, 1u, 0u}, rk);
  fluid_pair2_emit<4>(a.x, b.x, cl, emit);
  fluid_pair2_emit<5>(a.y, b.y, cl, emit);
  fluid_pair2_emit<6>(a.z, b.z, cl, emit);
  fluid_pair2_emit<7, false>(a.w, b.w, cl, emit);
}

// lb_collide for the two nodes of a thread (node, node + 1), lane by lane the same update:
// moments, relaxation and back-transform in packed arithmetic; the noise packed too
// (PACKED_NOISE: both nodes' Philox words turned into Gaussians together, fluid_noise2) or
// node by node.  Measured at L = 128: the packed noise cuts the warp instructions per 32 nodes
// from 541 to 483 and the 16-bit-storage step from 49.5 to 46.1 us, but holds two Philox
// states at once and slows the FP32-storage kernel (53.0 to 54.1 us), which waits on memory
// more than on issue slots; so FP32 storage takes the noise node by node.
template <bool DEV, bool NOISE, bool PACKED_NOISE>
__device__ __forceinline__ void lb_collide_pair(const f2 n[Q], f2 out[Q], const FluidK<float>& P,
                                                const RoundKeys& rk, unsigned long long* nonpos,
                                                const uint32_t step, const unsigned node) {
  f2 m[10];
  moments_0_9<f2>(n, m);
  const f2 rho = DEV ? f2(P.rho0) + m[0] : m[0];
  const f2 jx = m[1], jy = m[2], jz = m[3];
  const f2 ir(lb_rcp<float>(rho.v.x), lb_rcp<float>(rho.v.y));
  const f2 xx = jx * jx * ir, yy = jy * jy * ir, zz = jz * jz * ir;
  f2 a[Q];
  a[0] = m[0] * f2((float)(1.0 / 36.0));
  a[1] = jx * f2((float)(InvB<1>::v / 36.0));
  a[2] = jy * f2((float)(InvB<2>::v / 36.0));
  a[3] = jz * f2((float)(InvB<3>::v / 36.0));
  {
    const f2 e4 = xx + yy + zz, e5 = f2(2.0f) * xx - yy - zz, e6 = yy - zz;
    const f2 e7 = jx * jy * ir, e8 = jy * jz * ir, e9 = jx * jz * ir;
    a[4] = fma2(f2(P.wam[4]), m[4], f2(P.wae[4]) * e4);
    a[5] = fma2(f2(P.wam[5]), m[5], f2(P.wae[5]) * e5);
    a[6] = fma2(f2(P.wam[6]), m[6], f2(P.wae[6]) * e6);
    a[7] = fma2(f2(P.wam[7]), m[7], f2(P.wae[7]) * e7);
    a[8] = fma2(f2(P.wam[8]), m[8], f2(P.wae[8]) * e8);
    a[9] = fma2(f2(P.wam[9]), m[9], f2(P.wae[9]) * e9);
  }
#pragma unroll
  for (int k = 10; k < Q; ++k) a[k] = f2(0.0f);

  if (NOISE) {
    if (!(rho.v.x > 0.0f) || !(rho.v.y > 0.0f))
      atomicAdd(nonpos, (unsigned long long)(!(rho.v.x > 0.0f)) + (unsigned long long)(!(rho.v.y > 0.0f)));
    if constexpr (PACKED_NOISE) {
      // NoiseScale<float> of each lane: -2 ln(2) rho, a non-positive rho as 1e-30
      const f2 cl = f2(-1.38629436112f) * f2(rho.v.x > 0.0f ? rho.v.x : 1.0e-30f, rho.v.y > 0.0f ? rho.v.y : 1.0e-30f);
      fluid_noise2(step, node, rk, P.ncalls > 1, cl,
                   [&](int j, f2 g) { a[4 + j] = fma2(f2(P.wag[4 + j]), g, a[4 + j]); });
    } else {
      fluid_noise<float>(step, node, rk, P.ncalls > 1, NoiseScale<float>(rho.v.x),
                         [&](int j, float g) { a[4 + j].v.x = fmaf(P.wag[4 + j], g, a[4 + j].v.x); });
      fluid_noise<float>(step, node + 1, rk, P.ncalls > 1, NoiseScale<float>(rho.v.y),
                         [&](int j, float g) { a[4 + j].v.y = fmaf(P.wag[4 + j], g, a[4 + j].v.y); });
    }
  }

  if (P.body_on) {
    float d0[10], d1[10];
    force_moments(rho.v.x, jx.v.x, jy.v.x, jz.v.x, P.body_dJ[0], P.body_dJ[1], P.body_dJ[2], P.gs, P.gb, d0);
    force_moments(rho.v.y, jx.v.y, jy.v.y, jz.v.y, P.body_dJ[0], P.body_dJ[1], P.body_dJ[2], P.gs, P.gb, d1);
    a[1] = fma2(f2(d0[1], d1[1]), f2((float)(InvB<1>::v / 36.0)), a[1]);
    a[2] = fma2(f2(d0[2], d1[2]), f2((float)(InvB<2>::v / 36.0)), a[2]);
    a[3] = fma2(f2(d0[3], d1[3]), f2((float)(InvB<3>::v / 36.0)), a[3]);
    a[4] = fma2(f2(d0[4], d1[4]), f2((float)(InvB<4>::v / 36.0)), a[4]);
    a[5] = fma2(f2(d0[5], d1[5]), f2((float)(InvB<5>::v / 36.0)), a[5]);
    a[6] = fma2(f2(d0[6], d1[6]), f2((float)(InvB<6>::v / 36.0)), a[6]);
    a[7] = fma2(f2(d0[7], d1[7]), f2((float)(InvB<7>::v / 36.0)), a[7]);
    a[8] = fma2(f2(d0[8], d1[8]), f2((float)(InvB<8>::v / 36.0)), a[8]);
    a[9] = fma2(f2(d0[9], d1[9]), f2((float)(InvB<9>::v / 36.0)), a[9]);
  }

  pops_from_w2scaled<f2>(a, out);
}

template <class S, class R, bool DEV, bool NOISE, class I>
__device__ __forceinline__ void lb_collide_store(const R* n, S* __restrict__ dst, const FluidK<R>& P, const I pl,
                                                 const RoundKeys& rk, unsigned long long* nonpos,
                                                 const uint32_t step, const unsigned node,
                                                 const AngleTab* tab = nullptr) {
  R out[Q];
  lb_collide<R, DEV, NOISE>(n, out, P, rk, nonpos, step, node, tab);
#pragma unroll
  for (int i = 0; i < Q; ++i) st<S, R>(dst + ((I)i * pl + (I)node), out[i]);
}

// The 19 populations node (x, y, z) pulls from its neighbours in src (periodic): n_i(r) =
// src_i(r - c_i) (Sec. II B, Eq. 3, streaming).
template <class S, class R, class I>
__device__ __forceinline__ void lb_pull(const S* __restrict__ src, const unsigned L, const I pl, const unsigned x,
                                        const unsigned y, const unsigned z, R n[Q]) {
  const unsigned xm = x ? x - 1 : L - 1, xp = (x + 1 < L) ? x + 1 : 0;
  const unsigned ym = y ? y - 1 : L - 1, yp = (y + 1 < L) ? y + 1 : 0;
  const unsigned zm = z ? z - 1 : L - 1, zp = (z + 1 < L) ? z + 1 : 0;
  const unsigned LL = L * L;
  // row offsets of the source rows: [dy+1][dz+1] for a pull from y - dy, z - dz
  const unsigned ry[3] = {yp * L, y * L, ym * L};
  const unsigned rz[3] = {zp * LL, z * LL, zm * LL};
  const unsigned sxs[3] = {xp, x, xm};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const unsigned idx = sxs[cx(i) + 1] + ry[cy(i) + 1] + rz[cz(i) + 1];
    n[i] = ld<S, R>(src + ((I)i * pl + (I)idx));
  }
}

// Stage the previous step's corrections at the 19 pull sources of node (x, y, z) into
// col[i * stride] (shared memory).  A rolled loop with the directions unpacked from constants
// (this rare path must not raise the register count of the LB kernels), issuing asynchronous
// global-to-shared copies (cp.async) so that the 19 loads are in flight together; the
// calling thread waits for its own copies.
template <class R>
__device__ __forceinline__ void stage_corrections(const R* __restrict__ corr, unsigned long long plane, unsigned L,
                                                  unsigned x, unsigned y, unsigned z, R* col, unsigned stride) {
  static_assert(sizeof(R) == 4 || sizeof(R) == 8, "cp.async copies 4 or 8 bytes");
  constexpr unsigned long long PX = pack_component(0), PY = pack_component(1), PZ = pack_component(2);
#pragma unroll 1
  for (int i = 0; i < Q; ++i) {
    int sx = (int)x - unpack_component(PX, i), sy = (int)y - unpack_component(PY, i),
        sz = (int)z - unpack_component(PZ, i);
    sx = sx < 0 ? sx + (int)L : (sx >= (int)L ? sx - (int)L : sx);
    sy = sy < 0 ? sy + (int)L : (sy >= (int)L ? sy - (int)L : sy);
    sz = sz < 0 ? sz + (int)L : (sz >= (int)L ? sz - (int)L : sz);
    const unsigned idx = (unsigned)sx + L * ((unsigned)sy + L * (unsigned)sz);
    const unsigned dst = (unsigned)__cvta_generic_to_shared(col + i * stride);
    const R* src = corr + (unsigned long long)i * plane + idx;
    if (sizeof(R) == 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// One LB tile: pull-stream + collide for the (blockDim.x x blockDim.y) nodes at (tx, ty, z)
// (Sec. II B, Eq. 3).  Every thread loads its 19 populations and its mark word together; a
// node marked by the previous deferred step then stages that step's corrections at its pull
// sources (in shared memory, 19 x blockDim.x x blockDim.y values) and adds them to what it
// pulled, and one copy of the collision follows.  (Branching on the mark before the loads put
// an L2 round trip in front of every warp's loads, 1.4 us per launch at L = 128 with no node
// marked; with two inlined copies of the update, a warp holding marked and unmarked nodes
// ran both: 67.8 against 64.0 us with 1.5 % of the nodes marked.)
// CORR = false (a box without a chain): no correction code at all (the dead correction path
// alone cost 0.5 us per chained launch at L = 128).
template <class S, class R, bool DEV, bool NOISE, class I, bool CORR>
__device__ __forceinline__ void lb_tile(const S* __restrict__ src, S* __restrict__ dst, const FluidK<R>& P,
                                        const PendK<R>& Pd, const uint32_t step, unsigned tx, unsigned ty,
                                        unsigned z, R* stage, const AngleTab* tab) {
  const unsigned L = P.L;
  const unsigned x = tx * blockDim.x + threadIdx.x;
  const unsigned y = ty * blockDim.y + threadIdx.y;
  if (x >= L || y >= L) return;
  const unsigned node = x + L * (y + L * z);
  const unsigned mw = CORR && Pd.have_prev ? Pd.prev_mask[Pd.seg0 + (node >> kSegShift)] : 0u;
  const I pl = (I)P.plane;
  R n[Q];
  lb_pull<S, R, I>(src, L, pl, x, y, z, n);
  if (CORR && ((mw >> (node & 31u)) & 1u)) {
    const unsigned T = blockDim.x * blockDim.y, tid = threadIdx.x + blockDim.x * threadIdx.y;
    stage_corrections<R>(Pd.prev_dense, Pd.plane, L, x, y, z, stage + tid, T);
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] += stage[tid + i * T];
  }
  lb_collide_store<S, R, DEV, NOISE, I>(n, dst, P, pl, P.rk, P.nonpos, step, node, tab);
}

// Collide the pulled populations n0, n1 of the nodes (node, node + 1) and store the pairs
// (single precision: packed arithmetic for both nodes, lb_collide_pair; the noise packed
// too for 16-bit storage).
template <class S, class R, bool DEV, bool NOISE, class I>
__device__ __forceinline__ void lb_collide2_store(const R n0[Q], const R n1[Q], S* __restrict__ dst,
                                                  const FluidK<R>& P, const I pl, const RoundKeys& rk,
                                                  unsigned long long* nonpos, const uint32_t step,
                                                  const unsigned node) {
  if constexpr (sizeof(R) == 4) {
    f2 n[Q], o[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) n[i] = f2(n0[i], n1[i]);
    lb_collide_pair<DEV, NOISE, sizeof(S) == 2>(n, o, P, rk, nonpos, step, node);
#pragma unroll
    for (int i = 0; i < Q; ++i) st2<S, R>(dst + ((I)i * pl + (I)node), o[i].v.x, o[i].v.y);
  } else {
    R o0[Q], o1[Q];
    lb_collide<R, DEV, NOISE>(n0, o0, P, rk, nonpos, step, node);
    lb_collide<R, DEV, NOISE>(n1, o1, P, rk, nonpos, step, node + 1);
#pragma unroll
    for (int i = 0; i < Q; ++i) st2<S, R>(dst + ((I)i * pl + (I)node), o0[i], o1[i]);
  }
}

// The populations the two nodes (x0, y, z) and (x0 + 1, y, z), x0 even, pull from their
// neighbours (periodic; Sec. II B, Eq. 3): n0 for x0, n1 for x0 + 1.  The planes with c_x = 0
// read both nodes' sources with one two-element access (x0 even and L even keep it aligned);
// the planes with c_x = +-1 read their two sources x0 - c_x, x0 + 1 - c_x one by one.
template <class S, class R, class I>
__device__ __forceinline__ void lb_pull2(const S* __restrict__ src, const unsigned L, const I pl, const unsigned x0,
                                         const unsigned y, const unsigned z, R n0[Q], R n1[Q]) {
  const unsigned xm = x0 ? x0 - 1 : L - 1, xp = x0 + 1, xpp = (x0 + 2 < L) ? x0 + 2 : 0;
  const unsigned ym = y ? y - 1 : L - 1, yp = (y + 1 < L) ? y + 1 : 0;
  const unsigned zm = z ? z - 1 : L - 1, zp = (z + 1 < L) ? z + 1 : 0;
  const unsigned LL = L * L;
  const unsigned ry[3] = {yp * L, y * L, ym * L};
  const unsigned rz[3] = {zp * LL, z * LL, zm * LL};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const I row = (I)i * pl + (I)(ry[cy(i) + 1] + rz[cz(i) + 1]);
    if (cx(i) == 0) {
      ld2<S, R>(src + (row + (I)x0), n0[i], n1[i]);
    } else if (cx(i) == 1) {  // sources x0 - 1, x0
      n0[i] = ld<S, R>(src + (row + (I)xm));
      n1[i] = ld<S, R>(src + (row + (I)x0));
    } else {  // sources x0 + 1, x0 + 2
      n0[i] = ld<S, R>(src + (row + (I)xp));
      n1[i] = ld<S, R>(src + (row + (I)xpp));
    }
  }
}

// One LB tile with two nodes per thread along x (L even): the 2 blockDim.x x blockDim.y nodes
// at x = 2 (tx blockDim.x + threadIdx.x) + {0, 1}, y = ty blockDim.y + threadIdx.y, z.  The
// same update as lb_tile, node by node, with the 19 post-collision pairs written by
// two-element stores.  Marked nodes stage their corrections one node after the other into
// stage[tid + i * T], the same 19 T values as lb_tile.
template <class S, class R, bool DEV, bool NOISE, class I, bool CORR>
__device__ __forceinline__ void lb_tile2(const S* __restrict__ src, S* __restrict__ dst, const FluidK<R>& P,
                                         const PendK<R>& Pd, const uint32_t step, unsigned tx, unsigned ty,
                                         unsigned z, R* stage) {
  const unsigned L = P.L;
  const unsigned x0 = 2 * (tx * blockDim.x + threadIdx.x);
  const unsigned y = ty * blockDim.y + threadIdx.y;
  if (x0 >= L || y >= L) return;
  const unsigned node = x0 + L * (y + L * z);
  const unsigned mw = CORR && Pd.have_prev ? Pd.prev_mask[Pd.seg0 + (node >> kSegShift)] >> (node & 31u) : 0u;
  const I pl = (I)P.plane;
  R n0[Q], n1[Q];
  lb_pull2<S, R, I>(src, L, pl, x0, y, z, n0, n1);
  if (CORR && (mw & 3u)) {
    const unsigned T = blockDim.x * blockDim.y, tid = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll 1
    for (unsigned j = 0; j < 2; ++j) {
      if (!((mw >> j) & 1u)) continue;
      stage_corrections<R>(Pd.prev_dense, Pd.plane, L, x0 + j, y, z, stage + tid, T);
      if (j == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) n0[i] += stage[tid + i * T];
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) n1[i] += stage[tid + i * T];
      }
    }
  }
  lb_collide2_store<S, R, DEV, NOISE, I>(n0, n1, dst, P, pl, P.rk, P.nonpos, step, node);
}

// Programmatic dependent launch (a grid launched with programmatic stream serialization may
// start before the previous grid in the stream has completed): `wait` blocks until that
// previous grid has completed and its writes are visible; `release` lets the next grid start.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependent_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// LB kernel: 3D grid of (x-row segments) x (y rows) x z planes, plus (when it follows the
// bead kernel of its step) one more plane of blocks that only wait.  Every grid releases the
// next one at once.  Launched after the previous LB kernel (no chain): it waits for that grid
// before reading (P.pdl bit 0), so that only the launch latency and block scheduling overlap.
// Launched after the bead kernel of the same step: it reads nothing that kernel writes and
// runs beside it; the blocks of plane z = L, scheduled last, wait for it (bit 1), so that the
// grid completes only after the bead kernel and whatever comes next may take this grid's
// completion for both.  (A wait at the end of every block raised the register count.)
// Resident blocks of 256 threads per SM that the single-precision LB kernels are compiled
// for: 6 (40 registers) with one node per thread, 4 (64 registers) with two, so that 48 and 32
// warps keep 48 and 64 node updates' loads in flight per SM quarter; the FP64 kernel is
// bound by FP64 arithmetic and compiled without a bound.
template <class R, bool PAIR>
struct LbMinBlocks {
  static constexpr int value = sizeof(R) == 4 ? (PAIR ? 4 : 6) : 1;
};

// PAIR: two nodes per thread along x (lb_tile2, L even), else one (lb_tile).
template <class S, class R, bool DEV, bool NOISE, class I, bool CORR, bool PAIR>
__global__ void __launch_bounds__(256, LbMinBlocks<R, PAIR>::value) k_lb_step(const S* __restrict__ src, S* __restrict__ dst,
                                                  const FluidK<R> P, const PendK<R> Pd, const uint32_t step) {
  extern __shared__ __align__(16) unsigned char lsm[];
  if (blockIdx.z >= P.L) {  // a waiting block
    allow_dependent_launch();
    if (P.pdl & 2) grid_dependency_wait();
    return;
  }
  if (P.pdl & 1) grid_dependency_wait();
  allow_dependent_launch();
  const uint32_t k = launch_step(P, step);
  const AngleTab* tab = nullptr;
  if constexpr (sizeof(R) == 8) {
    __shared__ AngleTab s_tab;
    if (P.angle_tab) {  // before any thread leaves: every thread reaches the barrier
      fill_angle_tables(&s_tab, threadIdx.x + blockDim.x * threadIdx.y);
      __syncthreads();
      tab = &s_tab;
    }
  }
  if constexpr (PAIR)
    lb_tile2<S, R, DEV, NOISE, I, CORR>(src, dst, P, Pd, k, blockIdx.x, blockIdx.y, blockIdx.z,
                                        reinterpret_cast<R*>(lsm));
  else
    lb_tile<S, R, DEV, NOISE, I, CORR>(src, dst, P, Pd, k, blockIdx.x, blockIdx.y, blockIdx.z,
                                       reinterpret_cast<R*>(lsm), tab);
}

// ---------------------------------------------------------------------------------------
// bead / coupling kernel (one thread block or one cluster)
// ---------------------------------------------------------------------------------------
// cell of a coordinate: floor(x/a) mod L into [0, L); frac = x/a - floor(x/a)
template <class R>
__device__ __forceinline__ int cell_of(R x, R a, int L, R& frac) {
  const R s = x / a;
  const R f = floor(s);
  frac = s - f;
  long long c = (long long)f;
  long long r = c % L;
  if (r < 0) r += L;
  return (int)r;
}

// Pair vector r_b - r_j under the minimum image convention from compensated positions
// (hi in [0, box), lo): the coordinate above box/2 is moved down by the box, which is exact
// (Sterbenz), so the difference of two nearby beads carries no rounding from their distance to
// the origin.
template <class R>
__device__ __forceinline__ R pair_delta(R hb, R lb, R hj, R lj, R box, R half_box) {
  const R dh = hb - hj;
  if (dh > half_box)
    hb -= box;
  else if (dh < -half_box)
    hj -= box;
  return (hb - hj) + (lb - lj);
}

// FENE (bonded) + WCA force coefficient: force on b = coef * d
template <class R>
__device__ __forceinline__ R pair_coef(R r2, bool bonded, const ChainK<R>& C, unsigned* status) {
  R coef = R(0);
  if (r2 < C.rc2) {
    const R s2 = C.sig2 / r2;
    const R s6 = s2 * s2 * s2;
    coef += R(24) * C.eps / r2 * (R(2) * s6 * s6 - s6);
  }
  if (bonded) {
    if (r2 >= C.R0sq) {
      atomicOr(status, ST_FENE);
    } else {
      coef -= C.kfene / (R(1) - r2 / C.R0sq);
    }
  }
  return coef;
}

// Conservative forces (FENE + WCA + external) on the beads bb0 .. bb1-1 from the positions of
// all beads staged in shared memory; `lanes` threads per bead split the partners and combine
// in a fixed shuffle tree.
template <class R>
__device__ __forceinline__ void chain_forces_block(const R* __restrict__ sh, const R* __restrict__ sl,
                                                   const ChainK<R>& C, R* __restrict__ out, const int bb0,
                                                   const int bb1) {
  const int N = C.N, nt = blockDim.x * blockDim.y, tid = threadIdx.x + blockDim.x * threadIdx.y;
  int lanes = 1;
  while (lanes < 32 && lanes * 2 * (bb1 - bb0) <= nt) lanes *= 2;
  const int per = nt / lanes;
  const int lane = tid % lanes;
  for (int base = bb0; base < bb1; base += per) {
    const int b = base + tid / lanes;
    R f[3] = {R(0), R(0), R(0)};
    if (b < bb1) {
      for (int j = lane; j < N; j += lanes) {
        if (j == b) continue;
        const bool bonded = (j == b - 1) || (j == b + 1);
        R d[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
          d[q] = pair_delta<R>(sh[3 * b + q], sl[3 * b + q], sh[3 * j + q], sl[3 * j + q], C.box, C.half_box);
        const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const R coef = pair_coef<R>(r2, bonded, C, C.status);
        f[0] += coef * d[0];
        f[1] += coef * d[1];
        f[2] += coef * d[2];
      }
    }
    for (int o = lanes / 2; o > 0; o /= 2) {
#pragma unroll
      for (int q = 0; q < 3; ++q) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o, lanes);
    }
    if (b < bb1 && lane == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) out[3 * b + q] = f[q] + C.ext[q];
    }
  }
}

constexpr int kGroupHashMax = 1024;  // entries grouped by hash table (else sorted)

// Hash of a lattice node index onto a power-of-two table: the "lowbias32" integer finaliser
// (xor-shift-multiply constants from C. Wellons' hash prospector).  Lattice neighbours differ
// in few, structured bits, which a plain multiplicative hash maps to clustered low bits.
__device__ __forceinline__ unsigned hash_node(int node, unsigned mask) {
  unsigned h = (unsigned)node;
  h ^= h >> 16;
  h *= 0x7feb352du;
  h ^= h >> 15;
  h *= 0x846ca68bu;
  h ^= h >> 16;
  return h & mask;
}

// Bitonic sort (ascending) of M keys in shared memory, M a power of two >= 32, by a block of
// nt threads (a multiple of 32).  Compare-exchange distances j >= 32 go through shared memory
// with a barrier each; the distances j < 32 of every stage run in registers, each warp
// holding a contiguous chunk of 32 keys and exchanging through shuffles.
__device__ __forceinline__ void bitonic_sort_block(unsigned long long* keys, int M, int tid, int nt) {
  for (int k = 2; k <= M; k <<= 1) {
    for (int j = k >> 1; j >= 32; j >>= 1) {
      for (int i = tid; i < M; i += nt) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long ka = keys[i], kb = keys[ixj];
          const bool up = (i & k) == 0;
          if ((ka > kb) == up) {
            keys[i] = kb;
            keys[ixj] = ka;
          }
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < M; i += nt) {  // whole warps: M and nt are multiples of 32
      unsigned long long v = keys[i];
      const bool up = (i & k) == 0;
      for (int j = (k >> 1) < 16 ? (k >> 1) : 16; j > 0; j >>= 1) {
        const unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)v, j);
        const unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), j);
        const unsigned long long o = ((unsigned long long)hi << 32) | lo;
        // the lower element of the pair keeps the minimum in an ascending run
        const bool take_min = ((i & j) == 0) == up;
        v = take_min ? (o < v ? o : v) : (o > v ? o : v);
      }
      keys[i] = v;
    }
    __syncthreads();
  }
}

// post-stream populations at node (qx,qy,qz): rho and lattice momentum; with the dense field
// of the previous step's corrections (corr != nullptr) added to the pulled populations
template <class S, class R, bool DEV>
__device__ __forceinline__ void gather_node_c(const S* __restrict__ pop, const FluidK<R>& P, int qx, int qy,
                                              int qz, R mom[4], const R* __restrict__ corr) {
  const int L = (int)P.L;
  unsigned idx[Q];
  R v[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int sx = qx - cx(i), sy = qy - cy(i), sz = qz - cz(i);
    sx = sx < 0 ? sx + L : (sx >= L ? sx - L : sx);
    sy = sy < 0 ? sy + L : (sy >= L ? sy - L : sy);
    sz = sz < 0 ? sz + L : (sz >= L ? sz - L : sz);
    idx[i] = (unsigned)sx + (unsigned)L * ((unsigned)sy + (unsigned)L * (unsigned)sz);
    v[i] = ld<S, R>(pop + (unsigned long long)i * P.plane + idx[i]);
  }
  if (corr) {
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] += corr[(unsigned long long)i * P.plane + idx[i]];
  }
  R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rho += v[i];
    if (cx(i)) jx += R(cx(i)) * v[i];
    if (cy(i)) jy += R(cy(i)) * v[i];
    if (cz(i)) jz += R(cz(i)) * v[i];
  }
  mom[0] = DEV ? P.rho0 + rho : rho;
  mom[1] = jx;
  mom[2] = jy;
  mom[3] = jz;
}

// post-stream populations at node (qx,qy,qz): rho and lattice momentum
template <class S, class R, bool DEV>
__device__ __forceinline__ void gather_node(const S* __restrict__ pop, const FluidK<R>& P, int qx, int qy,
                                            int qz, R mom[4]) {
  const int L = (int)P.L;
  R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int sx = qx - cx(i), sy = qy - cy(i), sz = qz - cz(i);
    sx = sx < 0 ? sx + L : (sx >= L ? sx - L : sx);
    sy = sy < 0 ? sy + L : (sy >= L ? sy - L : sy);
    sz = sz < 0 ? sz + L : (sz >= L ? sz - L : sz);
    const unsigned idx = (unsigned)sx + (unsigned)L * ((unsigned)sy + (unsigned)L * (unsigned)sz);
    const R v = ld<S, R>(pop + (unsigned long long)i * P.plane + idx);
    rho += v;
    if (cx(i)) jx += R(cx(i)) * v;
    if (cy(i)) jy += R(cy(i)) * v;
    if (cz(i)) jz += R(cz(i)) * v;
  }
  mom[0] = DEV ? P.rho0 + rho : rho;
  mom[1] = jx;
  mom[2] = jy;
  mom[3] = jz;
}

// The pending correction of one node (the coupling of Sec. II B, spread back to the fluid): the sum
// of its entries' reactions in entry order (ent(base) .. ent(base + cnt - 1) ascending),
// turned into population corrections at pending-list index u, written to the list and the
// dense field, and the nodes pulling from it marked.
template <class R, class Ent>
__device__ __forceinline__ void node_correction(const FluidK<R>& P, const ChainK<R>& C, const PendK<R>& Pd, int L,
                                                int N, int u, int node, Ent ent, int base, int cnt) {
  const int e0 = ent(base);
  R f[3] = {R(0), R(0), R(0)};
  for (int r = base; r < base + cnt; ++r) {
    const int e = ent(r);
    const R w = C.e_w[e] * C.spread;
    const int sub = e / (8 * N), b = (e - sub * 8 * N) >> 3;
    const R* fch = C.fc_hist + sub * 3 * N;
    f[0] -= w * fch[3 * b + 0] * C.inv_a3;
    f[1] -= w * fch[3 * b + 1] * C.inv_a3;
    f[2] -= w * fch[3 * b + 2] * C.inv_a3;
  }
  const R rho = C.e_mom[e0], jx = C.e_mom[C.cap + e0], jy = C.e_mom[2 * C.cap + e0],
          jz = C.e_mom[3 * C.cap + e0];
  R dJ[3] = {f[0] * C.dJ_scale, f[1] * C.dJ_scale, f[2] * C.dJ_scale};
  R dm[10];
  if (P.body_on) {
    // the LB kernel applies the body-force correction on every node; here add the
    // difference between the correction for the total force and the body-only one
    R dmb[10];
    force_moments(rho, jx, jy, jz, P.body_dJ[0], P.body_dJ[1], P.body_dJ[2], P.gs, P.gb, dmb);
    force_moments(rho, jx, jy, jz, dJ[0] + P.body_dJ[0], dJ[1] + P.body_dJ[1], dJ[2] + P.body_dJ[2],
                  P.gs, P.gb, dm);
#pragma unroll
    for (int k = 0; k < 10; ++k) dm[k] -= dmb[k];
  } else {
    force_moments(rho, jx, jy, jz, dJ[0], dJ[1], dJ[2], P.gs, P.gb, dm);
  }
  R dn[Q];
  dmoments_to_dpops(dm, dn);
  const int pz = node / (L * L), py = (node / L) % L, px = node % L;
  Pd.cur_pos[u] = make_int4(node, px, py, pz);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    Pd.cur_dn[q * Pd.cap + u] = dn[q];
    Pd.cur_dense[(unsigned long long)q * Pd.plane + (unsigned)node] = dn[q];
  }
  if (Pd.mark) {  // mark the nodes that pull from this node
    // neighbour coordinates [c + 1] for c = -1, 0, +1 (periodic)
    const int xs[3] = {px ? px - 1 : L - 1, px, px + 1 < L ? px + 1 : 0};
    const int ys[3] = {py ? py - 1 : L - 1, py, py + 1 < L ? py + 1 : 0};
    const int zs[3] = {pz ? pz - 1 : L - 1, pz, pz + 1 < L ? pz + 1 : 0};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const unsigned idx = (unsigned)xs[cx(q) + 1] + (unsigned)L * ((unsigned)ys[cy(q) + 1] + (unsigned)L * (unsigned)zs[cz(q) + 1]);
      atomicOr(&Pd.cur_mask[Pd.seg0 + (idx >> kSegShift)], 1u << (idx & 31u));
    }
  }
}

// Clear the mask words of the nodes that pull from node (px, py, pz) (whole words: in its slot
// a word holds marks of one list only)
__device__ __forceinline__ void clear_marks(unsigned* mask, unsigned seg0, int L, int px, int py, int pz) {
  const int xs[3] = {px ? px - 1 : L - 1, px, px + 1 < L ? px + 1 : 0};
  const int ys[3] = {py ? py - 1 : L - 1, py, py + 1 < L ? py + 1 : 0};
  const int zs[3] = {pz ? pz - 1 : L - 1, pz, pz + 1 < L ? pz + 1 : 0};
  unsigned last = 0xffffffffu;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const unsigned idx = (unsigned)xs[cx(q) + 1] + (unsigned)L * ((unsigned)ys[cy(q) + 1] + (unsigned)L * (unsigned)zs[cz(q) + 1]);
    const unsigned w = seg0 + (idx >> kSegShift);
    if (w != last) mask[w] = 0u;
    last = w;
  }
}

// Generic address of the same shared-memory location in block 0 of the cluster
template <class T>
__device__ __forceinline__ const T* cluster_rank0(const T* p) {
  unsigned long long d;
  asm volatile("mapa.u64 %0, %1, 0;" : "=l"(d) : "l"(reinterpret_cast<unsigned long long>(p)));
  return reinterpret_cast<const T*>(d);
}

// Barrier over the thread blocks of a cluster; release/acquire order every memory access
// before it (shared, distributed shared and global) before every access after it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One coupled bead step for one chain: velocity Verlet, FENE/WCA, interpolation of the
// post-stream flow at the 8 corners, friction + Langevin force, and the deterministic
// spreading of the reaction into a list of per-node population corrections.  Run by one
// thread block (any size, multiple of 32), or by the G blocks of a cluster (rank: this
// block's): each block computes the drift of every bead into its shared memory and then
// takes a contiguous share of the beads (forces, corners and gathers, friction), of the old
// list (clearing) and of the new list's nodes (corrections); block 0 writes the positions
// and groups the corner entries by node in its shared memory, which the others read.
// Most of this work is scattered global memory traffic, which G blocks issue from G SMs.
// `smem` holds the positions (6N R; with G > 1 also the half-step velocities and image
// counters, 9N R + 3N int), later the node grouping table (or the sort keys, G = 1 only), as
// sized by the host.
template <class S, class R, bool DEV>
__device__ __forceinline__ void bead_step_block(const S* __restrict__ pop, const FluidK<R>& P, const ChainK<R>& C,
                                                const PendK<R>& Pd, const uint32_t step, unsigned char* smem,
                                                const int rank = 0, const int G = 1) {
  const int N = C.N;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y, nt = blockDim.x * blockDim.y;
  const int L = (int)P.L;
  const R h = C.h;
  R* sx = reinterpret_cast<R*>(smem);
  R* sl = sx + 3 * N;
  R* svh = sl + 3 * N;                             // G > 1: half-step velocities
  int* simg = reinterpret_cast<int*>(svh + 3 * N);  // G > 1: image counters
  const R* vhp = G > 1 ? svh : C.vh;
  const int b0 = rank * N / G, b1 = (rank + 1) * N / G;  // this block's beads
  // clear this slot's dense entries of its old list (two steps back, or already applied);
  // the new list overwrites the old one only in phase 5, after several barriers.  The threads
  // the first drift leaves idle (t >= 3N; every block drifts every bead) clear while the others
  // drift, so that the two chains of global round trips overlap; with no thread idle, every
  // thread clears first.
  {
    const int nd = 3 * N;
    const int c0 = nd < nt ? nd : 0, cn = nt - c0;  // the clearing threads [c0, nt)
    if (tid >= c0) {
      const int old = *Pd.cur_count;
      for (int u = (tid - c0) + rank * cn; u < old; u += G * cn) {
        const int4 p = Pd.cur_pos[u];
        R* d = Pd.cur_dense + (unsigned)p.x;
#pragma unroll
        for (int i = 0; i < Q; ++i) d[(unsigned long long)i * Pd.plane] = R(0);
        if (Pd.cur_mask) clear_marks(Pd.cur_mask, Pd.seg0, L, p.y, p.z, p.w);
      }
    }
  }
  const R* corr = Pd.have_prev ? Pd.prev_dense : nullptr;

  // MD substeps against the frozen post-stream fluid (one for LB step = MD step)
  for (int sub = 0; sub < C.nsub; ++sub) {
  const int eoff = sub * 8 * N;
  // 1. first half kick and drift: v_half = v + h F/2m, x' = x + h v_half, in compensated
  //    (hi, lo) arithmetic, then wrapped into [0, box) with the image counter
  const bool first = sub == 0;  // later substeps continue from the written state
  const R* const vin = first ? C.v_in : C.v;
  const R* const Fin = first ? C.F_in : C.F;
  const R* const xin = first ? C.x_in : C.x;
  const R* const xlin = first ? C.xl_in : C.xl;
  const int* const imgin = first ? C.img_in : C.img;
  for (int t = tid; t < 3 * N; t += nt) {
    const R vh = vin[t] + h * Fin[t] / (R(2) * C.m);
    const R dx = h * vh;
    const R xh = xin[t];
    R hi = xh + dx;
    const R bp = hi - xh;
    R lo = xlin[t] + ((xh - (hi - bp)) + (dx - bp));
    {
      const R s2 = hi + lo;
      lo = lo - (s2 - hi);
      hi = s2;
    }
    int im = imgin[t];
    if (hi < R(0)) {
      const R s2 = C.box + hi;
      lo += hi - (s2 - C.box);
      hi = s2;
      --im;
    }
    if (hi >= C.box) {
      hi -= C.box;
      ++im;
    }
    if (G == 1) {
      C.vh[t] = vh;
      C.x[t] = hi;
      C.xl[t] = lo;
      C.img[t] = im;
    } else {
      svh[t] = vh;
      simg[t] = im;
    }
    sx[t] = hi;
    sl[t] = lo;
  }
  __syncthreads();
  if (G > 1) {
    cluster_sync();  // every block has read the state of the previous (sub)step
    if (rank == 0)
      for (int t = tid; t < 3 * N; t += nt) {
        C.vh[t] = svh[t];
        C.x[t] = sx[t];
        C.xl[t] = sl[t];
        C.img[t] = simg[t];
      }
  }

  // 2. conservative forces at x': FENE on bonds, WCA on all pairs, minimum image
  chain_forces_block<R>(sx, sl, C, C.fcons, b0, b1);

  // 3. corners of the block's beads: cell, trilinear weight, post-stream rho and J at the node
  for (int e0 = 8 * b0 + tid; e0 < 8 * b1; e0 += nt) {
    const int b = e0 >> 3, c = e0 & 7, e = eoff + e0;
    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    R fr[3];
    int cl[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      R unused;
      const R xh = sx[3 * b + q];
      cl[q] = cell_of<R>(xh, C.a, L, unused);
      // fractional position inside the cell from the exact remainder xh - floor(xh/a) a
      const R f = floor(xh / C.a);
      fr[q] = (fma(-f, C.a, xh) + sl[3 * b + q]) / C.a;
    }
    const int qx = (cl[0] + dx) % L, qy = (cl[1] + dy) % L, qz = (cl[2] + dz) % L;
    const R w = (dx ? fr[0] : R(1) - fr[0]) * (dy ? fr[1] : R(1) - fr[1]) * (dz ? fr[2] : R(1) - fr[2]);
    R mom[4];
    gather_node_c<S, R, DEV>(pop, P, qx, qy, qz, mom, corr);
    C.e_node[e] = qx + L * (qy + L * qz);
    C.e_w[e] = w;
#pragma unroll
    for (int q = 0; q < 4; ++q) C.e_mom[q * C.cap + e] = mom[q];
  }
  __syncthreads();

  // 4. friction + Langevin force, second half kick
  for (int b = b0 + tid; b < b1; b += nt) {
    R ub[3] = {R(0), R(0), R(0)};
    for (int c = 0; c < 8; ++c) {
      const int e = eoff + 8 * b + c;
      const R w = C.e_w[e];
      const R ir = R(1) / C.e_mom[e];
      ub[0] += w * C.e_mom[1 * C.cap + e] * ir;
      ub[1] += w * C.e_mom[2 * C.cap + e] * ir;
      ub[2] += w * C.e_mom[3 * C.cap + e] * ir;
    }
    R g[4] = {R(0), R(0), R(0), R(0)};
    if (C.amp != R(0)) gauss4<R>(step * (uint32_t)C.nsub + (uint32_t)sub, (uint32_t)b, 0u, C.k0, C.k1, g);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int t = 3 * b + q;
      const R vh = vhp[t];
      const R fc = -C.zeta * (vh - ub[q] * C.u_scale) + C.amp * g[q];
      const R Ft = C.fcons[t] + fc;
      C.Fc[t] = fc;
      C.fc_hist[sub * 3 * N + t] = fc;
      C.F[t] = Ft;
      const R vn = vh + h * Ft / (R(2) * C.m);
      C.v[t] = vn;
      if (C.snap && sub == C.nsub - 1) {  // the step's end state, as the bead read-back forms it
        double* sn = C.snap + (size_t)(step & 1u) * 6 * N;
        const int im = G > 1 ? simg[t] : C.img[t];
        sn[t] = __dadd_rn(__dadd_rn((double)sx[t], (double)sl[t]), __dmul_rn((double)im, C.snap_box));
        sn[3 * N + t] = (double)vn;
      }
    }
  }
  __syncthreads();
  if (G > 1) cluster_sync();  // every bead is done
  }  // substeps

  // 5. deterministic spreading: group the corner entries by node, sum each node's
  //    contributions in entry order, then turn the node force into population corrections.
  //    Up to kGroupHashMax entries the grouping uses a hash table in shared memory; the
  //    table's slots number the nodes of the pending list (that order depends on the table
  //    layout; no value does).  Beyond, a bitonic sort of (node, entry) keys.
  const int ne = 8 * N * C.nsub;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  if (ne <= kGroupHashMax) {
    int H = 64;
    while (H < 2 * ne) H <<= 1;
    int* tkey = reinterpret_cast<int*>(smem);  // node of the slot, -1 = empty
    int* tcnt = tkey + H;                       // entries of the slot, then the fill cursor
    int* toff = tcnt + H;                       // first list position of the slot's entries
    int* lslot = toff + H;                      // slot of the u-th node of the pending list
    int* eslot = lslot + H;                     // slot of each entry
    int* elist = eslot + ne;                    // entries grouped by slot
    int* wsum = elist + ne;                     // scan scratch: 2 x 32 warp totals, node count
    if (rank == 0) {  // block 0 groups the entries
      for (int h = tid; h < H; h += nt) {
        tkey[h] = -1;
        tcnt[h] = 0;
      }
      __syncthreads();
      for (int e = tid; e < ne; e += nt) {
        const int node = C.e_node[e];
        unsigned h = hash_node(node, (unsigned)H - 1);
        for (int it = 0; it < H; ++it) {  // at most half full: a free slot or the node is found
          const int old = atomicCAS(&tkey[h], -1, node);
          if (old == -1 || old == node) break;
          h = (h + 1) & (unsigned)(H - 1);
        }
        eslot[e] = (int)h;
        atomicAdd(&tcnt[h], 1);
      }
      __syncthreads();
      // exclusive scans over the slots, in slot order: list offsets and node numbers.  Each
      // thread owns a contiguous run of slots; warp scans, then a scan of the warp totals.
      {
        const int per = (H + nt - 1) / nt;
        const int h0 = tid * per < H ? tid * per : H, h1 = h0 + per < H ? h0 + per : H;
        int sc = 0, sl = 0;
        for (int h = h0; h < h1; ++h) {
          sc += tcnt[h];
          sl += tcnt[h] > 0;
        }
        int ic = sc, il = sl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int yc = __shfl_up_sync(0xffffffffu, ic, o), yl = __shfl_up_sync(0xffffffffu, il, o);
          if (lane >= o) {
            ic += yc;
            il += yl;
          }
        }
        if (lane == 31) {
          wsum[warp] = ic;
          wsum[32 + warp] = il;
        }
        __syncthreads();
        if (warp == 0) {
          const int vc = lane < nwarp ? wsum[lane] : 0, vl = lane < nwarp ? wsum[32 + lane] : 0;
          int jc = vc, jl = vl;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int yc = __shfl_up_sync(0xffffffffu, jc, o), yl = __shfl_up_sync(0xffffffffu, jl, o);
            if (lane >= o) {
              jc += yc;
              jl += yl;
            }
          }
          if (lane < nwarp) {
            wsum[lane] = jc - vc;
            wsum[32 + lane] = jl - vl;
          }
          if (lane == 31) {
            *Pd.cur_count = jl;
            wsum[64] = jl;
          }
        }
        __syncthreads();
        int bc = wsum[warp] + ic - sc, bl = wsum[32 + warp] + il - sl;
        for (int h = h0; h < h1; ++h) {
          const int c = tcnt[h];
          toff[h] = bc;
          if (c > 0) lslot[bl] = h;
          tcnt[h] = bc;  // fill cursor
          bc += c;
          bl += c > 0;
        }
      }
      __syncthreads();
      for (int e = tid; e < ne; e += nt) elist[atomicAdd(&tcnt[eslot[e]], 1)] = e;
      __syncthreads();
      for (int u = tid; u < wsum[64]; u += nt) {  // each node's entries in entry order
        const int h = lslot[u];
        const int base = toff[h], cnt = tcnt[h] - base;
        for (int r = base + 1; r < base + cnt; ++r) {  // (insertion sort of a short list)
          const int e = elist[r];
          int q = r - 1;
          while (q >= base && elist[q] > e) {
            elist[q + 1] = elist[q];
            --q;
          }
          elist[q + 1] = e;
        }
      }
    }  // block 0
    __syncthreads();
    if (G > 1) cluster_sync();  // block 0's table is complete
    // the table of block 0, read by every block of the cluster (distributed shared memory)
    const int* tk = G > 1 ? cluster_rank0(tkey) : tkey;
    const int* to = G > 1 ? cluster_rank0(toff) : toff;
    const int* tc = G > 1 ? cluster_rank0(tcnt) : tcnt;
    const int* ls = G > 1 ? cluster_rank0(lslot) : lslot;
    const int* el = G > 1 ? cluster_rank0(elist) : elist;
    const int nnode = (G > 1 ? cluster_rank0(wsum) : wsum)[64];
    const int u0 = rank * nnode / G, u1 = (rank + 1) * nnode / G;  // this block's nodes
    for (int u = u0 + tid; u < u1; u += nt) {  // one thread per node, in list order
      const int h = ls[u];
      const int base = to[h], cnt = tc[h] - base;
      node_correction<R>(P, C, Pd, L, N, u, tk[h], [&](int r) { return el[r]; }, base, cnt);
    }
    if (G > 1) cluster_sync();  // block 0's table is read until here
  } else {  // (one block: the host launches G = 1 beyond kGroupHashMax entries)
    if (rank != 0) return;
    int M = 32;  // at least one warp-wide chunk; padding keys sort to the end
    while (M < ne) M <<= 1;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem);
    for (int i = tid; i < M; i += nt)
      keys[i] = (i < ne) ? (((unsigned long long)(unsigned)C.e_node[i] << 32) | (unsigned)i) : ~0ull;
    __syncthreads();
    bitonic_sort_block(keys, M, tid, nt);
    // leaders: first entry of each node run, numbered in order (chunks of 32 entries: each
    // warp counts the leaders of its chunks, warp 0 scans the chunk counts)
    int* slot = reinterpret_cast<int*>(keys + M);
    int* cbase = slot + ne;
    const int nchunk = (ne + 31) >> 5;
    for (int c = warp; c < nchunk; c += nwarp) {
      const int i = (c << 5) + lane;
      const int lead = i < ne && ((i == 0) || ((keys[i] >> 32) != (keys[i - 1] >> 32)));
      const unsigned mask = __ballot_sync(0xffffffffu, lead);
      if (lane == 0) cbase[c] = __popc(mask);
    }
    __syncthreads();
    if (warp == 0) {
      int base = 0;
      for (int c0 = 0; c0 < nchunk; c0 += 32) {
        const int c = c0 + lane;
        const int v = c < nchunk ? cbase[c] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (c < nchunk) cbase[c] = base + incl - v;
        base += __shfl_sync(0xffffffffu, incl, 31);
      }
      if (lane == 0) *Pd.cur_count = base;
    }
    __syncthreads();
    for (int c = warp; c < nchunk; c += nwarp) {
      const int i = (c << 5) + lane;
      const int lead = i < ne && ((i == 0) || ((keys[i] >> 32) != (keys[i - 1] >> 32)));
      const unsigned mask = __ballot_sync(0xffffffffu, lead);
      if (i < ne) slot[i] = lead ? cbase[c] + __popc(mask & ((1u << lane) - 1u)) : -1;
    }
    __syncthreads();
    for (int i = tid; i < ne; i += nt) {
      const int u = slot[i];
      if (u < 0) continue;
      const int node = (int)(keys[i] >> 32);
      int cnt = 1;
      while (i + cnt < ne && (int)(keys[i + cnt] >> 32) == node) ++cnt;
      node_correction<R>(P, C, Pd, L, N, u, node, [&](int r) { return (int)(keys[r] & 0xffffffffu); }, i, cnt);
    }
  }
}

// The bead step as its own grid.  Launched with programmatic stream serialization
// after the previous step's LB kernel (which completes only after the previous bead kernel),
// it waits for that grid before reading; then it releases the LB kernel of the same step,
// which reads neither its outputs nor anything it writes and runs alongside.
// The grid is one cluster of G blocks (G = 1: a single block).
template <class S, class R, bool DEV>
__global__ void __launch_bounds__(512) k_bead_step(const S* __restrict__ pop, const FluidK<R> P,
                                                    const ChainK<R> C, const PendK<R> Pd, const uint32_t step) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned rank, G;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(G));
  grid_dependency_wait();
  allow_dependent_launch();
  bead_step_block<S, R, DEV>(pop, P, C, Pd, launch_step(P, step), smem, (int)rank, (int)G);
}

// B[i][node] += dn_i at every pending node (each node appears once in the list), and the
// applied entries of the dense correction field and the list's mask words (mask may be null)
// back to zero; one thread per (node, population): blockIdx.y is the population
template <class S, class R>
__global__ void __launch_bounds__(256) k_apply_pending(S* __restrict__ pop, const FluidK<R> P,
                                                        const int4* __restrict__ p_pos,
                                                        const R* __restrict__ p_dn,
                                                        const int* __restrict__ p_count, int cap,
                                                        R* __restrict__ dense, unsigned* __restrict__ mask,
                                                        unsigned seg0) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= *p_count) return;
  const int i = blockIdx.y;
  const int4 p = p_pos[u];
  const unsigned long long off = (unsigned long long)i * P.plane + (unsigned)p.x;
  st<S, R>(pop + off, ld<S, R>(pop + off) + p_dn[i * cap + u]);
  dense[off] = R(0);
  if (mask && i == 0) clear_marks(mask, seg0, (int)P.L, p.y, p.z, p.w);
}

// one trajectory frame: unwrapped positions x + xl + img * box in FP64, in the order (and
// without contraction) of the host read-back
template <class R>
__global__ void k_record_frame(const R* __restrict__ x, const R* __restrict__ xl, const int* __restrict__ img,
                               int n3, double box, double* __restrict__ dst) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += gridDim.x * blockDim.x)
    dst[t] = __dadd_rn(__dadd_rn((double)x[t], (double)xl[t]), __dmul_rn((double)img[t], box));
}

// bead read-back: out[0..n3) unwrapped positions as k_record_frame forms them, out[n3..2 n3)
// velocities, FP64
template <class R>
__global__ void k_bead_readback(const R* __restrict__ x, const R* __restrict__ xl, const int* __restrict__ img,
                                const R* __restrict__ v, int n3, double box, double* __restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n3; t += gridDim.x * blockDim.x) {
    out[t] = __dadd_rn(__dadd_rn((double)x[t], (double)xl[t]), __dmul_rn((double)img[t], box));
    out[n3 + t] = (double)v[t];
  }
}

// ---------------------------------------------------------------------------------------
// initial state, conversions, reductions
// ---------------------------------------------------------------------------------------
template <class S, class R, bool DEV>
__global__ void k_init_rest(S* __restrict__ pop, unsigned long long nnodes, unsigned long long plane, R rho0) {
  const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if (t >= nnodes) return;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const R v = DEV ? R(0) : rho0 * (R(w36(i)) / R(36));
    st<S, R>(pop + (unsigned long long)i * plane + t, v);
  }
}

// one population plane: full FP64 values <-> storage
// planes p0 .. p0 + gridDim.y - 1 of the stored populations as full FP64 populations:
// dst[(i - p0) n + t] = n_i(t) (+ w_i rho0 for deviation storage); dst may be page-locked host
// memory the device addresses directly
template <class S, class R, bool DEV>
__global__ void __launch_bounds__(256) k_planes_to_f64(double* __restrict__ dst, const S* __restrict__ src,
                                                       unsigned long long n, unsigned long long plane, int p0,
                                                       double rho0) {
  const int i = p0 + (int)blockIdx.y;
  const double wr = DEV ? rho0 * (double)w36(i) / 36.0 : 0.0;
  const S* s = src + (unsigned long long)i * plane;
  double* d = dst + (unsigned long long)blockIdx.y * n;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x)
  {
    const double v = (double)ld<S, R>(s + t);
    d[t] = DEV ? v + wr : v;
  }
}
// the inverse: planes p0 .. p0 + gridDim.y - 1 of the stored populations from FP64 src
template <class S, class R, bool DEV>
__global__ void __launch_bounds__(256) k_planes_from_f64(S* __restrict__ dst, const double* __restrict__ src,
                                                         unsigned long long n, unsigned long long plane, int p0,
                                                         double rho0) {
  const int i = p0 + (int)blockIdx.y;
  const double wr = DEV ? rho0 * (double)w36(i) / 36.0 : 0.0;
  S* d = dst + (unsigned long long)i * plane;
  const double* s = src + (unsigned long long)blockIdx.y * n;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x)
    st<S, R>(d + t, (R)(DEV ? s[t] - wr : s[t]));
}

// per-block FP64 partial sums of (sum n, Jx, Jy, Jz) of the stored populations
template <class S, class R, bool DEV>
__global__ void __launch_bounds__(256) k_fluid_partials(const S* __restrict__ pop, unsigned long long nnodes,
                                                         unsigned long long plane, double* __restrict__ part) {
  const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  double v[4] = {0, 0, 0, 0};
  if (t < nnodes) {
    R r = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R n = ld<S, R>(pop + (unsigned long long)i * plane + t);
      r += n;
      if (cx(i)) jx += R(cx(i)) * n;
      if (cy(i)) jy += R(cy(i)) * n;
      if (cz(i)) jz += R(cz(i)) * n;
    }
    v[0] = (double)r;
    v[1] = (double)jx;
    v[2] = (double)jy;
    v[3] = (double)jz;
  }
  __shared__ double sh[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double a = v[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double a = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[threadIdx.x][w];
    part[4ull * blockIdx.x + threadIdx.x] = a;
  }
}

// observables: fluid sums from the partials, bead quantities from the chain state (FP64)
template <class R>
struct ObsK {
  const double* part;
  int nparts;
  double mass_rest;   // rho0 L^3 for deviation storage (0 for full storage)
  double a3, u_scale;  // a^3, a/h
  int N;
  const R* x;
  const R* xl;
  const int* img;
  const R* v;
  const R* Fc;
  double box, m, h;
  const double* xref;  // 3N reference positions
  double* acc;         // [samples, sum Rg2, sum Re2]
  const unsigned long long* nonpos;
  double* out;         // LB_NOBS values
  long long step;
  int accumulate;      // 1: add this sample to the accumulators
};

template <class R>
__global__ void __launch_bounds__(256) k_observables(const ObsK<R> O) {
  __shared__ double sh[16][8];
  const int tid = threadIdx.x;
  // fluid: fixed-order reduction of the partials
  double f[4] = {0, 0, 0, 0};
  for (int p = tid; p < O.nparts; p += blockDim.x)
    for (int q = 0; q < 4; ++q) f[q] += O.part[4ll * p + q];
  // beads
  double cm[3] = {0, 0, 0}, mv[3] = {0, 0, 0}, fc[3] = {0, 0, 0}, v2 = 0;
  for (int b = tid; b < O.N; b += blockDim.x) {
    for (int q = 0; q < 3; ++q) {
      const double xu = (double)O.x[3 * b + q] + (double)O.xl[3 * b + q] + (double)O.img[3 * b + q] * O.box;
      cm[q] += xu;
      const double vv = (double)O.v[3 * b + q];
      mv[q] += O.m * vv;
      v2 += vv * vv;
      fc[q] += (double)O.Fc[3 * b + q];
    }
  }
  double vals[14] = {f[0], f[1], f[2], f[3], cm[0], cm[1], cm[2], mv[0], mv[1], mv[2], fc[0], fc[1], fc[2], v2};
  for (int q = 0; q < 14; ++q) {
    double a = vals[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((tid & 31) == 0) sh[q][tid >> 5] = a;
  }
  __syncthreads();
  __shared__ double tot[14];
  if (tid < 14) {
    double a = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[tid][w];
    tot[tid] = a;
  }
  __syncthreads();
  // second pass: R_g^2 about the centre of mass, R_e^2, MSDs
  const int N = O.N;
  double rg = 0;
  for (int b = tid; b < N; b += blockDim.x) {
    for (int q = 0; q < 3; ++q) {
      const double xu = (double)O.x[3 * b + q] + (double)O.xl[3 * b + q] + (double)O.img[3 * b + q] * O.box;
      const double d = xu - tot[4 + q] / N;
      rg += d * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) rg += __shfl_down_sync(0xffffffffu, rg, o);
  __syncthreads();
  if ((tid & 31) == 0) sh[15][tid >> 5] = rg;
  __syncthreads();
  if (tid == 0) {
    double rgt = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) rgt += sh[15][w];
    double* o = O.out;
    o[0] = (double)O.step;
    o[1] = (O.mass_rest + tot[0]) * O.a3;
    const double s = O.u_scale * O.a3;
    o[5] = tot[1] * s;
    o[6] = tot[2] * s;
    o[7] = tot[3] * s;
    o[2] = o[5] + tot[7] + 0.5 * O.h * tot[10];
    o[3] = o[6] + tot[8] + 0.5 * O.h * tot[11];
    o[4] = o[7] + tot[9] + 0.5 * O.h * tot[12];
    double Rg2 = 0, Re2 = 0, g1 = 0, g3 = 0;
    if (N > 0) {
      Rg2 = rgt / N;
      double cmr[3] = {0, 0, 0};
      for (int b = 0; b < N; ++b)
        for (int q = 0; q < 3; ++q) cmr[q] += O.xref[3 * b + q];
      const int i0 = (N - 1) / 2, i1 = N / 2;
      for (int q = 0; q < 3; ++q) {
        const double xe = (double)O.x[3 * (N - 1) + q] + (double)O.xl[3 * (N - 1) + q] + (double)O.img[3 * (N - 1) + q] * O.box;
        const double xs = (double)O.x[q] + (double)O.xl[q] + (double)O.img[q] * O.box;
        Re2 += (xe - xs) * (xe - xs);
        const double a0 = (double)O.x[3 * i0 + q] + (double)O.xl[3 * i0 + q] + (double)O.img[3 * i0 + q] * O.box - O.xref[3 * i0 + q];
        const double a1 = (double)O.x[3 * i1 + q] + (double)O.xl[3 * i1 + q] + (double)O.img[3 * i1 + q] * O.box - O.xref[3 * i1 + q];
        g1 += 0.5 * (a0 * a0 + a1 * a1);
        const double dc = (tot[4 + q] - cmr[q]) / N;
        g3 += dc * dc;
      }
      o[10] = tot[4] / N;
      o[11] = tot[5] / N;
      o[12] = tot[6] / N;
      o[15] = O.m * tot[13] / (3.0 * N);
    } else {
      o[10] = o[11] = o[12] = 0;
      o[15] = 0;
    }
    o[8] = Rg2;
    o[9] = Re2;
    o[13] = g1;
    o[14] = g3;
    o[16] = (double)*O.nonpos;
    if (O.accumulate) {
      O.acc[0] += 1.0;
      O.acc[1] += Rg2;
      O.acc[2] += Re2;
    }
    o[17] = O.acc[0];
    o[18] = O.acc[0] > 0 ? O.acc[1] / O.acc[0] : 0.0;
    o[19] = O.acc[0] > 0 ? O.acc[2] / O.acc[0] : 0.0;
  }
}

}  // namespace gblb

namespace gblb {

// Forces of the initial configuration: F = F_cons(x0) (+ external), F_c = 0.
template <class R>
__global__ void __launch_bounds__(512) k_chain_init_forces(const ChainK<R> C) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sx = reinterpret_cast<R*>(smem);
  R* sl = sx + 3 * C.N;
  for (int t = threadIdx.x; t < 3 * C.N; t += blockDim.x) {
    sx[t] = C.x[t];
    sl[t] = C.xl[t];
  }
  __syncthreads();
  chain_forces_block<R>(sx, sl, C, C.F, 0, C.N);
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * C.N; t += blockDim.x) C.Fc[t] = R(0);
}

}  // namespace gblb
