// Adjoint (reverse-mode derivative) of the coupled LB + chain step with the noise held
// fixed, for gradients of a chain observable with respect to the initial bead positions and
// the friction coefficient zeta.
//
// The forward step (see lb_device.cuh) is, per step k:
//   beads:  v_h = v + h F/2m;  x' = x + h v_h;  F_cons(x');  u_b = sum_c w_c(x') J_c/rho_c (a/h);
//           F_c = -zeta (v_h - u_b) + sqrt(2 kT zeta / h) g_b;  F' = F_cons + F_c;
//           v' = v_h + h F'/2m
//   fluid:  n_ps = pull-stream(n*);  n*' = collide(n_ps) + correction(rho, J, f(x', F_c))
// The adjoint runs the same chain of maps backwards: the fluid adjoint lambda(n*) goes
// through the transposed collision Jacobian (node-local) and the push-stream (the transpose
// of the pull); the chain adjoint through the transposed Jacobians of the integrator, the
// friction, the interpolation (including the gradient of the trilinear weights), the
// spreading and force correction, and the Hessian of FENE + WCA.  The bead side produces the
// derivative with respect to (rho, J) of the post-stream state at the <= 8N corner nodes,
// which a small kernel adds into the pushed fluid adjoint.
#pragma once
#include "lb_device.cuh"

namespace gblb {

// dcoef/d(r^2) of the pair force coefficient (force on b = coef * d, see pair_coef)
template <class R>
__device__ __forceinline__ R pair_coef_deriv(R r2, bool bonded, const ChainK<R>& C) {
  R dc = R(0);
  if (r2 < C.rc2) {
    const R s2 = C.sig2 / r2;
    const R s6 = s2 * s2 * s2;
    dc += R(24) * C.eps / (r2 * r2) * (R(-14) * s6 * s6 + R(4) * s6);
  }
  if (bonded && r2 < C.R0sq) {
    const R t = R(1) - r2 / C.R0sq;
    dc -= C.kfene / C.R0sq / (t * t);
  }
  return dc;
}

// xbar_b += sum_j [coef I + 2 coef' d d^T] (Fbar_b - Fbar_j): the chain-force Hessian applied
// to the force adjoint.  Positions in shared memory (hi, lo); lanes per bead as in
// chain_forces_block; the result is added to out.
template <class R>
__device__ __forceinline__ void chain_force_vjp_block(const R* __restrict__ sh, const R* __restrict__ sl,
                                                      const R* __restrict__ fbar, const ChainK<R>& C,
                                                      R* __restrict__ out) {
  const int N = C.N, nt = blockDim.x, tid = threadIdx.x;
  int lanes = 1;
  while (lanes < 32 && lanes * 2 * N <= nt) lanes *= 2;
  const int per = nt / lanes;
  const int lane = tid % lanes;
  for (int base = 0; base < N; base += per) {
    const int b = base + tid / lanes;
    R acc[3] = {R(0), R(0), R(0)};
    if (b < N) {
      for (int j = lane; j < N; j += lanes) {
        if (j == b) continue;
        R d[3], D[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          d[q] = pair_delta<R>(sh[3 * b + q], sl[3 * b + q], sh[3 * j + q], sl[3 * j + q], C.box, C.half_box);
          D[q] = fbar[3 * b + q] - fbar[3 * j + q];
        }
        const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const bool bonded = (j == b - 1) || (j == b + 1);
        const R c = pair_coef<R>(r2, bonded, C, C.status);
        const R cp = pair_coef_deriv<R>(r2, bonded, C);
        const R dD = d[0] * D[0] + d[1] * D[1] + d[2] * D[2];
#pragma unroll
        for (int q = 0; q < 3; ++q) acc[q] += c * D[q] + R(2) * cp * dD * d[q];
      }
    }
    for (int o = lanes / 2; o > 0; o /= 2) {
#pragma unroll
      for (int q = 0; q < 3; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o, lanes);
    }
    if (b < N && lane == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) out[3 * b + q] += acc[q];
    }
  }
}

// Vector-Jacobian product of force_moments with respect to (rho, J, dJ).
template <class R>
__device__ __forceinline__ void force_moments_vjp(R rho, R jx, R jy, R jz, R dx, R dy, R dz, R gs, R gb,
                                                  const R dmb[10], R& rhob, R Jb[3], R dJb[3]) {
  const R ir = R(1) / rho;
  const R ux = (jx + R(0.5) * dx) * ir, uy = (jy + R(0.5) * dy) * ir, uz = (jz + R(0.5) * dz) * ir;
  const R cs = R(0.5) * (R(1) + gs);
  const R cdiag = (R(1) + gb) / R(3) - R(2) / R(3) * cs;
  const R Pxx = dmb[4] + R(2) * dmb[5];
  const R Pyy = dmb[4] - dmb[5] + dmb[6];
  const R Pzz = dmb[4] - dmb[5] - dmb[6];
  const R Pxy = dmb[7], Pyz = dmb[8], Pxz = dmb[9];
  const R udb = cdiag * (Pxx + Pyy + Pzz);
  // adjoint of U'
  const R Ux = R(2) * cs * dx * Pxx + cs * (dy * Pxy + dz * Pxz) + udb * dx;
  const R Uy = R(2) * cs * dy * Pyy + cs * (dx * Pxy + dz * Pyz) + udb * dy;
  const R Uz = R(2) * cs * dz * Pzz + cs * (dy * Pyz + dx * Pxz) + udb * dz;
  // adjoint of dJ: direct (modes 1..3), through the stress products, through U'
  dJb[0] = dmb[1] + R(2) * cs * ux * Pxx + cs * (uy * Pxy + uz * Pxz) + udb * ux + R(0.5) * Ux * ir;
  dJb[1] = dmb[2] + R(2) * cs * uy * Pyy + cs * (ux * Pxy + uz * Pyz) + udb * uy + R(0.5) * Uy * ir;
  dJb[2] = dmb[3] + R(2) * cs * uz * Pzz + cs * (uy * Pyz + ux * Pxz) + udb * uz + R(0.5) * Uz * ir;
  Jb[0] = Ux * ir;
  Jb[1] = Uy * ir;
  Jb[2] = Uz * ir;
  rhob = -(ux * Ux + uy * Uy + uz * Uz) * ir;
}

// a-bar_k = sum_i w_i e_k(c_i) nbar_i: adjoint of the scaled moments from the adjoint of
// the populations they produce (n_i = w_i sum_k e_k(c_i) a_k)
template <class R>
__device__ __forceinline__ void scaled_moment_adjoint(const R nb[Q], R ab[Q]) {
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    R acc = R(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int c = basis(k, i) * w36(i);
      if (c != 0) acc += R(c) * nb[i];
    }
    ab[k] = acc * (R(1) / R(36));
  }
}

// ---------------------------------------------------------------------------------------
// fluid adjoint of one step: lambda(n*_k) from lambda(n*_{k+1}), every node
//   n_ps(r) = pull(n*_k) ; n*_{k+1}(r) = collide(n_ps(r))   (corrections handled sparsely)
//   nbar_ps(r) = J_collide(r)^T lambda_{k+1}(r);  lambda_k,i(r - e_i) = nbar_ps,i(r)   (push)
// ---------------------------------------------------------------------------------------
// Launched with programmatic stream serialization after the previous reverse step's bead
// adjoint: it waits for that grid (which has added its forced-node terms to lam_in) before
// reading, then releases the bead adjoint of its own step, which runs beside it (see
// k_adj_bead).
template <class S, class R, bool DEV, bool NOISE>
__global__ void __launch_bounds__(256) k_adj_lb(const S* __restrict__ state, const R* __restrict__ lam_in,
                                                 R* __restrict__ lam_out, const FluidK<R> P, const uint32_t step_arg) {
  grid_dependency_wait();
  allow_dependent_launch();
  const uint32_t step = launch_step(P, step_arg);
  const unsigned L = P.L;
  const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned y = blockIdx.y * blockDim.y + threadIdx.y;
  const unsigned z = blockIdx.z;
  if (x >= L || y >= L) return;
  const unsigned node = x + L * (y + L * z);
  unsigned nb_idx[Q];  // node r - e_i: source of the pull, target of the push
  R n[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const unsigned sx = (x + L - (unsigned)(cx(i) + 0)) % L;
    const unsigned sy = (y + L - (unsigned)(cy(i) + 0)) % L;
    const unsigned sz = (z + L - (unsigned)(cz(i) + 0)) % L;
    nb_idx[i] = sx + L * (sy + L * sz);
    n[i] = ld<S, R>(state + (unsigned long long)i * P.plane + nb_idx[i]);
  }
  R m[10];
  moments_0_9<R>(n, m);
  const R rho = DEV ? P.rho0 + m[0] : m[0];
  const R jx = m[1], jy = m[2], jz = m[3];
  const R ir = R(1) / rho;
  R lb_[Q], ab[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) lb_[i] = lam_in[(unsigned long long)i * P.plane + node];
  scaled_moment_adjoint<R>(lb_, ab);
  // m-bar from the scaled-moment map a(m)
  R mb[10];
  mb[0] = ab[0];
  mb[1] = ab[1] * R(InvB<1>::v);
  mb[2] = ab[2] * R(InvB<2>::v);
  mb[3] = ab[3] * R(InvB<3>::v);
  R Eb[10];
#pragma unroll
  for (int k = 4; k < 10; ++k) {
    mb[k] = P.am[k] * ab[k];
    Eb[k] = P.ae[k] * ab[k];
  }
  const R E4 = (jx * jx + jy * jy + jz * jz) * ir, E5 = (R(2) * jx * jx - jy * jy - jz * jz) * ir;
  const R E6 = (jy * jy - jz * jz) * ir, E7 = jx * jy * ir, E8 = jy * jz * ir, E9 = jx * jz * ir;
  mb[0] -= (Eb[4] * E4 + Eb[5] * E5 + Eb[6] * E6 + Eb[7] * E7 + Eb[8] * E8 + Eb[9] * E9) * ir;
  mb[1] += (R(2) * jx * Eb[4] + R(4) * jx * Eb[5] + jy * Eb[7] + jz * Eb[9]) * ir;
  mb[2] += (R(2) * jy * Eb[4] - R(2) * jy * Eb[5] + R(2) * jy * Eb[6] + jx * Eb[7] + jz * Eb[8]) * ir;
  mb[3] += (R(2) * jz * Eb[4] - R(2) * jz * Eb[5] - R(2) * jz * Eb[6] + jy * Eb[8] + jx * Eb[9]) * ir;
  if (NOISE && rho > R(0)) {
    // a_k += ag_k sqrt(rho) g_k:  d/drho = ag_k g_k / (2 sqrt(rho))
    R acc = R(0);
    fluid_noise<R>(step, node, P.rk, P.ncalls > 1, NoiseScale<R>(R(1)),
                   [&](int j, R g) { acc += P.ag[4 + j] * g * ab[4 + j]; });
    mb[0] += acc * R(0.5) / sqrt(rho);
  }
  // nbar_ps,i = sum_k e_k(c_i) mb_k, pushed to r - e_i
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    R acc = R(0);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      const int c = basis(k, i);
      if (c != 0) acc += R(c) * mb[k];
    }
    lam_out[(unsigned long long)i * P.plane + nb_idx[i]] = acc;
  }
}

// Chain part of the adjoint of one step, one thread block.
// In:  bead state of step k (C.x/xl/img/v/F hold it), post-collision populations n*_k
//      (`state`), lambda(n*_{k+1}) (`lam`), xbar/vbar/fbar of step k+1.
// Out: xbar/vbar/fbar of step k (in place), zbar (+= d/dzeta), and lambda(n*_k) (`lam_out`)
//      completed: lambda_k,i(r - e_i) += rho-bar(r) + c_i . J-bar(r) at the forced nodes r.
// Launched with programmatic stream serialization after k_adj_lb of the same step, which writes
// the rest of lambda(n*_k): everything up to that last addition runs beside it, and the
// addition waits for it.
template <class R>
struct AdjK {
  R *xbar, *vbar, *fbar;  // 3N each, in/out across the reverse steps (global)
  double* zbar;           // accumulated d objective / d zeta (global)
  // scratch of one reverse step: carved from the kernel's dynamic shared memory at byte
  // offset smem_off when smem_scratch is set (small chains), else global memory
  R *vh, *ub, *g, *fc, *fct, *vhb, *xpb;  // 3N each
  R* e_gw;      // 3 x 8N weight gradients (per unit length)
  R* e_rb;      // 4 x 8N (rho-bar, J-bar) per entry
  R* u_fb;      // 3 x cap: f-bar per unique node
  R* u_rb;      // 4 x cap: forced-node (rho, J) adjoint per unique node
  R* u_sp;      // 4 x cap: (rho-bar, J-bar) summed per unique forced node
  R* zb_b;      // N: zeta-bar per bead
  R* ce_w;      // 8N: trilinear weight of each corner entry
  R* ce_mom;    // 4 x 8N: post-stream rho and J at each entry's node
  int* e_slot;  // 8N: unique-node slot of each entry
  int* u_node;  // cap: the unique forced nodes
  int* ce_node; // 8N: node of each corner entry
  int smem_scratch;
  unsigned smem_off;
};

// Carve the per-step scratch of AdjK from one region starting at base (16-byte aligned pieces,
// in a fixed order); returns its size.  base may be null to compute the size only.
template <class R>
__host__ __device__ inline size_t carve_adj_scratch(AdjK<R>& A, unsigned char* base, int N, int cap) {
  size_t off = 0;
  auto piece = [&](size_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += (bytes + 15) / 16 * 16;
    return p;
  };
  const size_t n3 = 3 * (size_t)N, ne = (size_t)cap;
  A.vh = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.ub = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.g = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.fc = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.fct = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.vhb = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.xpb = reinterpret_cast<R*>(piece(n3 * sizeof(R)));
  A.e_gw = reinterpret_cast<R*>(piece(3 * ne * sizeof(R)));
  A.e_rb = reinterpret_cast<R*>(piece(4 * ne * sizeof(R)));
  A.u_fb = reinterpret_cast<R*>(piece(3 * ne * sizeof(R)));
  A.u_rb = reinterpret_cast<R*>(piece(4 * ne * sizeof(R)));
  A.u_sp = reinterpret_cast<R*>(piece(4 * ne * sizeof(R)));
  A.zb_b = reinterpret_cast<R*>(piece((size_t)N * sizeof(R)));
  A.ce_w = reinterpret_cast<R*>(piece(ne * sizeof(R)));
  A.ce_mom = reinterpret_cast<R*>(piece(4 * ne * sizeof(R)));
  A.e_slot = reinterpret_cast<int*>(piece(ne * sizeof(int)));
  A.u_node = reinterpret_cast<int*>(piece(ne * sizeof(int)));
  A.ce_node = reinterpret_cast<int*>(piece(ne * sizeof(int)));
  return off;
}

template <class S, class R, bool DEV>
__global__ void __launch_bounds__(512) k_adj_bead(const S* __restrict__ state, const R* __restrict__ lam,
                                                   R* __restrict__ lam_out, const FluidK<R> P, const ChainK<R> C,
                                                   const AdjK<R> A0, const uint32_t step_arg) {
  const uint32_t step = launch_step(P, step_arg);
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = C.N, tid = threadIdx.x, nt = blockDim.x, L = (int)P.L;
  AdjK<R> A = A0;
  if (A0.smem_scratch) carve_adj_scratch(A, smem + A0.smem_off, N, C.cap);
  const R h = C.h;
  R* sx = reinterpret_cast<R*>(smem);
  R* sl = sx + 3 * N;
  // d/dzeta so far, read now so that the update at the end is a plain store (no other grid
  // writes it while this one runs: the previous reverse step has completed)
  const double zbar_in = tid == 0 ? *A.zbar : 0.0;
  // ---- forward recomputation of step k ------------------------------------------------
  for (int t = tid; t < 3 * N; t += nt) {
    const R vh = C.v[t] + h * C.F[t] / (R(2) * C.m);
    const R dx = h * vh;
    const R xh = C.x[t];
    R hi = xh + dx;
    const R bp = hi - xh;
    R lo = C.xl[t] + ((xh - (hi - bp)) + (dx - bp));
    {
      const R s2 = hi + lo;
      lo = lo - (s2 - hi);
      hi = s2;
    }
    if (hi < R(0)) {
      const R s2 = C.box + hi;
      lo += hi - (s2 - C.box);
      hi = s2;
    }
    if (hi >= C.box) hi -= C.box;
    A.vh[t] = vh;
    sx[t] = hi;
    sl[t] = lo;
  }
  __syncthreads();
  for (int e = tid; e < 8 * N; e += nt) {
    const int b = e >> 3, c = e & 7;
    const int d3[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    R fr[3];
    int cl[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      R unused;
      const R xh = sx[3 * b + q];
      cl[q] = cell_of<R>(xh, C.a, L, unused);
      const R f = floor(xh / C.a);
      fr[q] = (fma(-f, C.a, xh) + sl[3 * b + q]) / C.a;
    }
    R ws[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) ws[q] = d3[q] ? fr[q] : R(1) - fr[q];
    const R w = ws[0] * ws[1] * ws[2];
    // dw/dx_q = (+-1/a) * product of the other two factors
    A.e_gw[0 * C.cap + e] = (d3[0] ? R(1) : R(-1)) * ws[1] * ws[2] / C.a;
    A.e_gw[1 * C.cap + e] = (d3[1] ? R(1) : R(-1)) * ws[0] * ws[2] / C.a;
    A.e_gw[2 * C.cap + e] = (d3[2] ? R(1) : R(-1)) * ws[0] * ws[1] / C.a;
    const int qx = (cl[0] + d3[0]) % L, qy = (cl[1] + d3[1]) % L, qz = (cl[2] + d3[2]) % L;
    R mom[4];
    gather_node<S, R, DEV>(state, P, qx, qy, qz, mom);
    A.ce_node[e] = qx + L * (qy + L * qz);
    A.ce_w[e] = w;
#pragma unroll
    for (int q = 0; q < 4; ++q) A.ce_mom[q * C.cap + e] = mom[q];
  }
  __syncthreads();
  for (int b = tid; b < N; b += nt) {
    R ub[3] = {R(0), R(0), R(0)};
    for (int c = 0; c < 8; ++c) {
      const int e = 8 * b + c;
      const R w = A.ce_w[e], ir = R(1) / A.ce_mom[e];
      ub[0] += w * A.ce_mom[C.cap + e] * ir;
      ub[1] += w * A.ce_mom[2 * C.cap + e] * ir;
      ub[2] += w * A.ce_mom[3 * C.cap + e] * ir;
    }
    R g[4] = {R(0), R(0), R(0), R(0)};
    if (C.amp != R(0)) gauss4<R>(step, (uint32_t)b, 0u, C.k0, C.k1, g);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int t = 3 * b + q;
      const R u = ub[q] * C.u_scale;
      A.ub[t] = u;
      A.g[t] = g[q];
      A.fc[t] = -C.zeta * (A.vh[t] - u) + C.amp * g[q];
      // adjoint of the total force of step k+1 and of v_h (from v' = v_h + h F'/2m)
      A.fct[t] = A.fbar[t] + h / (R(2) * C.m) * A.vbar[t];
      A.vhb[t] = A.vbar[t];
      A.xpb[t] = A.xbar[t];  // x' is the position output of this step
    }
  }
  __syncthreads();
  // ---- unique forced nodes (same deterministic sort as the forward step) ----------------
  const int ne = 8 * N;
  int M = 1;
  while (M < ne) M <<= 1;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(smem + 6 * N * sizeof(R) + 16);
  keys = reinterpret_cast<unsigned long long*>((reinterpret_cast<uintptr_t>(keys) + 15) & ~(uintptr_t)15);
  for (int i = tid; i < M; i += nt)
    keys[i] = (i < ne) ? (((unsigned long long)(unsigned)A.ce_node[i] << 32) | (unsigned)i) : ~0ull;
  __syncthreads();
  if (ne <= nt) {
    // few entries: each thread places its key by its rank among all keys (distinct: the entry
    // index is in the low bits), two barriers instead of the bitonic network's log2(M)^2 / 2
    const unsigned long long mine = tid < ne ? keys[tid] : 0ull;
    int rank = 0;
    if (tid < ne)
      for (int j = 0; j < ne; ++j) rank += keys[j] < mine;
    __syncthreads();
    if (tid < ne) keys[rank] = mine;
    __syncthreads();
  } else {
    for (int k = 2; k <= M; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
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
    }
  }
  int* slot = reinterpret_cast<int*>(keys + M);
  __shared__ int s_nu;  // number of unique forced nodes
  if (tid < 32) {
    int base = 0;
    for (int c0 = 0; c0 < ne; c0 += 32) {
      const int i = c0 + tid;
      int lead = 0;
      if (i < ne) lead = (i == 0) || ((keys[i] >> 32) != (keys[i - 1] >> 32));
      const unsigned mask = __ballot_sync(0xffffffffu, lead);
      if (i < ne) slot[i] = lead ? base + __popc(mask & ((1u << tid) - 1u)) : -1;
      base += __popc(mask);
    }
    if (tid == 0) s_nu = base;
  }
  __syncthreads();
  // per unique node p: forward force density f(p), force-correction adjoint -> fbar(p),
  // forced-node (rho, J) adjoint; entry -> slot map
  for (int i = tid; i < ne; i += nt) {
    const int u = slot[i];
    if (u < 0) continue;
    const int node = (int)(keys[i] >> 32);
    const int e0 = (int)(keys[i] & 0xffffffffu);
    R f[3] = {R(0), R(0), R(0)};
    for (int r = i; r < ne && (int)(keys[r] >> 32) == node; ++r) {
      const int e = (int)(keys[r] & 0xffffffffu);
      const int b = e >> 3;
      A.e_slot[e] = u;
      f[0] -= A.ce_w[e] * A.fc[3 * b + 0] * C.inv_a3;
      f[1] -= A.ce_w[e] * A.fc[3 * b + 1] * C.inv_a3;
      f[2] -= A.ce_w[e] * A.fc[3 * b + 2] * C.inv_a3;
    }
    const R rho = A.ce_mom[e0], jx = A.ce_mom[C.cap + e0], jy = A.ce_mom[2 * C.cap + e0], jz = A.ce_mom[3 * C.cap + e0];
    R nb[Q], ab[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) nb[q] = lam[(unsigned long long)q * P.plane + (unsigned)node];
    scaled_moment_adjoint<R>(nb, ab);
    R dmb[10];
    dmb[0] = R(0);
    dmb[1] = ab[1] * R(InvB<1>::v);
    dmb[2] = ab[2] * R(InvB<2>::v);
    dmb[3] = ab[3] * R(InvB<3>::v);
    dmb[4] = ab[4] * R(InvB<4>::v);
    dmb[5] = ab[5] * R(InvB<5>::v);
    dmb[6] = ab[6] * R(InvB<6>::v);
    dmb[7] = ab[7] * R(InvB<7>::v);
    dmb[8] = ab[8] * R(InvB<8>::v);
    dmb[9] = ab[9] * R(InvB<9>::v);
    R rb, Jb[3], dJb[3];
    force_moments_vjp<R>(rho, jx, jy, jz, f[0] * C.dJ_scale, f[1] * C.dJ_scale, f[2] * C.dJ_scale, P.gs, P.gb, dmb,
                         rb, Jb, dJb);
    A.u_fb[u] = dJb[0] * C.dJ_scale;
    A.u_fb[C.cap + u] = dJb[1] * C.dJ_scale;
    A.u_fb[2 * C.cap + u] = dJb[2] * C.dJ_scale;
    A.u_rb[u] = rb;
    A.u_rb[C.cap + u] = Jb[0];
    A.u_rb[2 * C.cap + u] = Jb[1];
    A.u_rb[3 * C.cap + u] = Jb[2];
  }
  __syncthreads();
  // ---- per bead: spreading, friction, interpolation adjoints ---------------------------
  for (int b = tid; b < N; b += nt) {
    R fcb[3] = {A.fct[3 * b], A.fct[3 * b + 1], A.fct[3 * b + 2]};
    R fc[3] = {A.fc[3 * b], A.fc[3 * b + 1], A.fc[3 * b + 2]};
    R xpb[3] = {R(0), R(0), R(0)};
    // spreading: f(p) = -sum_e w_e F_c,b / a^3
    R wb[8];
    for (int c = 0; c < 8; ++c) {
      const int e = 8 * b + c, u = A.e_slot[e];
      const R fbx = A.u_fb[u], fby = A.u_fb[C.cap + u], fbz = A.u_fb[2 * C.cap + u];
      const R w = A.ce_w[e];
      fcb[0] -= w * C.inv_a3 * fbx;
      fcb[1] -= w * C.inv_a3 * fby;
      fcb[2] -= w * C.inv_a3 * fbz;
      wb[c] = -C.inv_a3 * (fc[0] * fbx + fc[1] * fby + fc[2] * fbz);
    }
    // friction + noise: F_c = -zeta (v_h - u_b) + amp(zeta) g
    R Ub[3], zb = R(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int t = 3 * b + q;
      A.vhb[t] -= C.zeta * fcb[q];
      Ub[q] = C.zeta * fcb[q];
      const R damp = C.zeta > R(0) ? C.amp / (R(2) * C.zeta) : R(0);
      zb += fcb[q] * (-(A.vh[t] - A.ub[t]) + damp * A.g[t]);
    }
    A.zb_b[b] = zb;
    // interpolation: u_b = sum_e w_e J_e / rho_e (a/h)
    for (int c = 0; c < 8; ++c) {
      const int e = 8 * b + c;
      const R w = A.ce_w[e], rho = A.ce_mom[e], ir = R(1) / rho;
      const R J[3] = {A.ce_mom[C.cap + e], A.ce_mom[2 * C.cap + e], A.ce_mom[3 * C.cap + e]};
      R ue[3], uJ = R(0);
#pragma unroll
      for (int q = 0; q < 3; ++q) ue[q] = J[q] * ir * C.u_scale;
      wb[c] += ue[0] * Ub[0] + ue[1] * Ub[1] + ue[2] * Ub[2];
      R ueb[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        ueb[q] = w * Ub[q];
        uJ += J[q] * ueb[q];
      }
      A.e_rb[e] = -C.u_scale * uJ * ir * ir;
#pragma unroll
      for (int q = 0; q < 3; ++q) A.e_rb[(q + 1) * C.cap + e] = C.u_scale * ueb[q] * ir;
      // trilinear weight gradient
#pragma unroll
      for (int q = 0; q < 3; ++q) xpb[q] += wb[c] * A.e_gw[q * C.cap + e];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) A.xpb[3 * b + q] += xpb[q];
  }
  __syncthreads();
  // ---- chain forces: x'bar += Hessian . F_cons-bar (F_cons-bar = F_total-bar) ---------
  chain_force_vjp_block<R>(sx, sl, A.fct, C, A.xpb);
  __syncthreads();
  // ---- integrator: x' = x + h v_h ; v_h = v + h F / 2m ------------------------------------
  for (int t = tid; t < 3 * N; t += nt) {
    const R xpb = A.xpb[t];
    const R vhb = A.vhb[t] + h * xpb;
    A.xbar[t] = xpb;
    A.vbar[t] = vhb;
    A.fbar[t] = h / (R(2) * C.m) * vhb;
  }
  // ---- sparse (rho, J) adjoint per unique node, entries summed in entry order -----------
  for (int i = tid; i < ne; i += nt) {
    const int u = slot[i];
    if (u < 0) continue;
    const int node = (int)(keys[i] >> 32);
    R v[4] = {A.u_rb[u], A.u_rb[C.cap + u], A.u_rb[2 * C.cap + u], A.u_rb[3 * C.cap + u]};
    for (int r = i; r < ne && (int)(keys[r] >> 32) == node; ++r) {
      const int e = (int)(keys[r] & 0xffffffffu);
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] += A.e_rb[q * C.cap + e];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) A.u_sp[q * C.cap + u] = v[q];
    A.u_node[u] = node;
  }
  // ---- zeta-bar: fixed-order block sum ----------------------------------------------------
  __syncthreads();
  if (tid == 0) {
    double acc = 0.0;
    for (int b = 0; b < N; ++b) acc += (double)A.zb_b[b];
    *A.zbar = zbar_in + acc;
  }
  // ---- lambda_k,i(r - e_i) += rho-bar(r) + c_i . J-bar(r) at the forced nodes, once the
  //      adjoint LB kernel of this step has written lambda_k (each (i, r - e_i) target belongs
  //      to one forced node r, so the additions do not collide) --------------------------
  //      In chunks of kAddBatch targets per thread: all loads of a chunk, then its stores (one
  //      memory round trip per chunk instead of one per target).
  grid_dependency_wait();
  const int nu = s_nu, total = Q * nu;
  constexpr int kAddBatch = 8;
  for (int k0 = tid; k0 < total; k0 += kAddBatch * nt) {
    unsigned long long at[kAddBatch];
    R v[kAddBatch], old[kAddBatch];
#pragma unroll
    for (int j = 0; j < kAddBatch; ++j) {
      const int k = k0 + j * nt;
      if (k >= total) break;
      const int i = k / nu, u = k - i * nu;
      const int node = A.u_node[u];
      const int x = node % L, y = (node / L) % L, z = node / (L * L);
      const int ex = unpack_component(pack_component(0), i), ey = unpack_component(pack_component(1), i),
                ez = unpack_component(pack_component(2), i);
      const int sx = (x - ex + L) % L, sy = (y - ey + L) % L, sz = (z - ez + L) % L;
      v[j] = A.u_sp[u] + R(ex) * A.u_sp[C.cap + u] + R(ey) * A.u_sp[2 * C.cap + u] + R(ez) * A.u_sp[3 * C.cap + u];
      at[j] = (unsigned long long)i * P.plane + (unsigned)(sx + L * (sy + L * sz));
      old[j] = lam_out[at[j]];
    }
#pragma unroll
    for (int j = 0; j < kAddBatch; ++j) {
      if (k0 + j * nt >= total) break;
      lam_out[at[j]] = old[j] + v[j];
    }
  }
}

// xbar += Hessian(F_cons)(x) . fbar at a given configuration (the initial force F_0 =
// F_cons(x_0) depends on x_0)
template <class R>
__global__ void __launch_bounds__(512) k_chain_force_vjp(const ChainK<R> C, const R* __restrict__ fbar,
                                                          R* __restrict__ xbar) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sx = reinterpret_cast<R*>(smem);
  R* sl = sx + 3 * C.N;
  for (int t = threadIdx.x; t < 3 * C.N; t += blockDim.x) {
    sx[t] = C.x[t];
    sl[t] = C.xl[t];
  }
  __syncthreads();
  chain_force_vjp_block<R>(sx, sl, fbar, C, xbar);
}

}  // namespace gblb
