/*
 * dg_internal.h -- internal state of the DG library shared by the host setup
 * (dg_host.cpp) and the CUDA kernels (dg_kernels.cu).  Not part of the ABI.
 */
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dg.h"

namespace dg {

constexpr int M = 4;          // conserved variables (rho, rho u, rho v, E)
constexpr int PMAX = 5;

// Geometry record of one element (8 doubles, 64 bytes):
//   jt[0..3] = J^tau = det J * J^{-1} in row-major order, so that the reference
//   flux is G_r = jt0 F1 + jt1 F2, G_s = jt2 F1 + jt3 F2; then 1/det J, det J.
constexpr int GEO = 8;

// Face record: left element, its local face, right element, its local face; on a
// boundary face r is the boundary code (DG_BC_WALL, DG_BC_STATE) and R = -1.
struct FaceConn { int32_t l, L, r, R; };
// Face geometry (8 doubles): unit normal n (left -> right) and half length l
// (Eq. len); then the products the edge flux uses, formed once on the host with
// h = l / 2: hk = h^2 gamma (gamma - 1), the scaled normal s = h n, and (gamma - 1) s.
struct FaceGeo { double nx, ny, hl, hk, sx, sy, gsx, gsy; };

struct DevTables {
  // All float64, device.  NP modes, NQ volume points, NF = 3*NE face points.
  double *BvT;   // [NP][NQ]   phi_j(r_k)                    (interpolation)
  double *Dr;    // [NQ][NP]   w_k d phi_j/dr (r_k)           (projection)
  double *Ds;    // [NQ][NP]   w_k d phi_j/ds (r_k)
  double *Lf;    // [NF][NP]   omega_k phi_j(r_{q,k})         (lifting)
  double *BfT;   // [NP][NF]   phi_j(r_{q,k})                 (edge traces)
  double *Pw;    // [NQ][NP]   w_k phi_j(r_k)                 (L2 projection of data)
  double *vr, *vs;   // [NQ] reference volume points
  // Sum factorisation on the collapsed grid (point k = ib*ND + ia, weight
  // w_k = wa(ia) wb(ib) / 8):
  //   phi_j(alpha_ia, beta_ib) = P_a(alpha_ia) chi_j(beta_ib),  a = a(j)
  double *SPa;   // [ND][ND]   P_a(alpha_ia)                 (Legendre, standard normalisation)
  double *SPaW;  // [ND][ND]   wa(ia) P_a(alpha_ia)
  double *SdPaW; // [ND][ND]   wa(ia) P_a'(alpha_ia)
  double *SChi;  // [NP][ND]   chi_j(beta_ib) = N_ab ((1-beta)/2)^a P_b^{(2a+1,0)}(beta)
  double *SChiA; // [NP][ND]   chi_j(beta_ib) wb(ib) / (4 (1 - s_ib))
  double *SdChiB;// [NP][ND]   chi_j'(beta_ib) wb(ib) / 4
  double *SHalf; // [ND]       (1 + alpha_ia) / 2
  // Sum factorisation on the edges (Gauss-Legendre nodes xi_k, weights omega_k):
  double *EChi;  // [NP][NE]   chi_j(xi_k)
  double *EWChi; // [NP][NE]   omega_k chi_j(xi_k)
  double *EWPa;  // [ND][NE]   omega_k P_a(xi_k)
  double *EChiM1;// [NP]       chi_j(-1)
  double *EPa;   // [ND][NE]   P_a(xi_k)
};

// One Runge-Kutta stage update of the element kernels (their mode 1), with
// R = R(c) the right-hand side of the stage input c:
//   out  = a0 u0 + b0 c + g dt R
//   out2 = x acc + y out + w dt R      (only when out2 is not null; acc may be out2)
// The SSP methods in Shu-Osher form use g = b0, i.e. out = a0 u0 + b0 (c + dt R),
// and no out2; the classical RK4 keeps the running sum of its stage derivatives
// in out2.
struct StageUpdate {
  double dt, a0, b0, g;
  const double *acc;
  double *out2;
  double x, y, w;
};
__host__ __device__ inline StageUpdate shu_osher(double dt, double a0, double b0) {
  return StageUpdate{dt, a0, b0, b0, nullptr, nullptr, 0.0, 0.0, 0.0};
}

// Stage i (0-based) of one step of the Runge-Kutta method `method` (dg_rk_method)
// on the state c, the stage buffer S and the classical RK4's running sum A: the
// element stage reads cin (and u0) and writes out with the update su.
//   SSP-RK3: u1 = c + dt L(c);  u2 = 3/4 c + 1/4 (u1 + dt L(u1)), over u1;
//            c <- 1/3 c + 2/3 (u2 + dt L(u2))
//   RK2 (Heun, Shu-Osher form): u1 = c + dt L(c);  c <- 1/2 c + 1/2 (u1 + dt L(u1))
//   RK4 with the running sum A of dt b_i k_i:
//     stage 1: S = c + dt/2 k1,  A = S - dt/3 k1   (= c + dt/6 k1)
//     stage 2: S = c + dt/2 k2,  A += dt/3 k2
//     stage 3: S = c + dt k3,    A += dt/3 k3
//     stage 4: c = A + dt/6 k4
// The host launches the stages one by one; the fused small-mesh stepper runs
// them inside one kernel.
struct RkStage {
  const double *cin, *u0;
  double *out;
  StageUpdate su;
};
__host__ __device__ inline int rk_num_stages(int method) {
  return method == DG_RK2 ? 2 : (method == DG_RK4 ? 4 : 3);
}
__host__ __device__ inline RkStage rk_stage(int method, int i, double dt, double *c, double *S, double *A) {
  if (method == DG_RK4) {
    if (i == 0) return RkStage{c, nullptr, S, StageUpdate{dt, 0.0, 1.0, 0.5, nullptr, A, 0.0, 1.0, -1.0 / 3.0}};
    if (i == 1) return RkStage{S, c, S, StageUpdate{dt, 1.0, 0.0, 0.5, A, A, 1.0, 0.0, 1.0 / 3.0}};
    if (i == 2) return RkStage{S, c, S, StageUpdate{dt, 1.0, 0.0, 1.0, A, A, 1.0, 0.0, 1.0 / 3.0}};
    return RkStage{S, A, c, StageUpdate{dt, 1.0, 0.0, 1.0 / 6.0, nullptr, nullptr, 0.0, 0.0, 0.0}};
  }
  if (method == DG_RK2) {
    if (i == 0) return RkStage{c, nullptr, S, shu_osher(dt, 0.0, 1.0)};
    return RkStage{S, c, c, shu_osher(dt, 0.5, 0.5)};
  }
  if (i == 0) return RkStage{c, nullptr, S, shu_osher(dt, 0.0, 1.0)};
  if (i == 1) return RkStage{S, c, S, shu_osher(dt, 0.75, 0.25)};
  return RkStage{S, c, c, shu_osher(dt, 1.0 / 3.0, 2.0 / 3.0)};
}

// Which devices a one-time setting of a kernel (cudaFuncSetAttribute, a per-device
// property) has been applied on: bit d for device d < 64; larger device numbers
// apply it on every launch.
struct PerDevice {
  std::atomic<unsigned long long> done{0};
  bool test(int dev) const { return dev >= 0 && dev < 64 && ((done.load() >> dev) & 1ull); }
  void set(int dev) {
    if (dev >= 0 && dev < 64) done.fetch_or(1ull << dev);
  }
};

// Per-kernel CUDA-event timing (dg_set_timing / dg_kernel_times).
struct Timing {
  bool on = false;
  struct Rec { cudaEvent_t a, b; int kind; };
  std::vector<Rec> pool;        // event pairs, reused
  size_t used = 0;              // pairs recorded since the last harvest
  double ms[DG_NKINDS] = {};
  int64_t launches[DG_NKINDS] = {};
};

// A CUDA graph of several Runge-Kutta steps, captured once per (state pointer,
// dt, precision, method, step count) and replayed by dg_rk_step on an internal
// stream.
struct GraphCache {
  cudaStream_t stream = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
  cudaGraphExec_t exec = nullptr;
  double *c = nullptr;
  double dt = 0.0;
  int prec = -1, steps = 0, method = -1;
  bool broken = false;        // capture failed once: use plain launches from then on
};

}  // namespace dg

struct dg_mesh {
  int p, np, nq, nd, ne;
  int rule;               // dg_vol_rule: the collapsed grid or the symmetric rule
  double gamma;
  int64_t N, F;
  int64_t Fb;                  // boundary faces (the first Fb of the face list)
  int64_t n_state_faces;       // boundary faces with a prescribed state
  bool bstate_set;             // dg_set_boundary_state was called (or none is needed)
  double *bstate;              // [Fb][ne][M] prescribed boundary states (device)
  double *bxy;                 // [Fb][ne][2] boundary points (device)
  int device;
  int num_sms;
  // device arrays
  double *geo;                 // [N][GEO]
  double *xy;                  // [N][6]
  int32_t *elem_face;          // [N][3]: f*2 + side (0 = left, 1 = right)
  int32_t *elem_nbr;           // [N][3]: the element across each local face
  dg::FaceConn *face_conn;     // [F]: the Fb boundary faces first (r = boundary code < 0)
  dg::FaceGeo *face_geo;       // [F]
  dg::DevTables tab;
  double *table_block;         // one allocation holding every table
  size_t table_doubles;
  // work buffers
  double *trace;               // [N][3*ne][M]
  double *fhat;                // [F][ne][M]
  double *stage;               // [N][M][np]
  double *host_state;          // [N][M][np] device copy used by dg_rk_step_host
  double *rk_acc;              // [N][M][np] running sum of the RK4 stages (first RK4 call)
  double *partial;             // [nblk][M] totals partials
  int *err_flag;               // device int: bit 0 = a bounded tensor-core wait expired,
                               //             bit 1 = a non-physical state was met
  double rin_min;              // smallest inscribed radius 2 area / perimeter
  double phi1;                 // the constant basis function (sqrt 2)
  int limiter;                 // dg_set_limiter: limit every stage (p = 1, float64)
  double *totals_dev;          // [M]
  int totals_blocks;
  // scratch for the adjoint (allocated on first use)
  double *adj_buf;
  size_t adj_doubles;
  dg::Timing *timing;
  dg::GraphCache *graph;
  unsigned *gbar;              // [2] grid barrier of the fused small-mesh stepper (count, generation)
  unsigned char *tc_img[2];    // B operand images of the tensor-core kernel (1xTF32, 3xTF32)
  int small_stepper;           // dg_set_small_mesh_stepper (on by default)
  cudaStream_t copy_stream;    // dg_rk_step_host's copies out (created on first use)
  cudaEvent_t copy_ev[2];
};

namespace dg {

// Kernel launchers (dg_kernels.cu).  All return a cudaError_t cast to int.
// copy (optional): also writes c to copy (c may be host memory the device reaches)
int launch_traces(const dg_mesh *m, const double *c, double *trace, void *stream, double *copy = nullptr);
int launch_face_flux(const dg_mesh *m, const double *trace, double *fhat, void *stream);
int resident_grid(const dg_mesh *m, const void *kernel, int threads, int64_t n, int *per_sm);
// out = mode==0 ? R(c) : the stage update su (and su.out2);  trace_out may be null.
// Elements [e0, e1) only (e1 < 0: all; the same bits per element either way).
int launch_element(const dg_mesh *m, const double *c, const double *u0, double *out,
                   double *trace_out, const double *fhat, const StageUpdate &su, int mode, void *stream,
                   int64_t e0 = 0, int64_t e1 = -1);
// The float64 element kernel's resident wave: tiles (all SMs) and elements per tile.
int element_wave(const dg_mesh *m, int *tiles, int *elems_per_tile);
// out = mode==0 ? R(c) : a0*u0 + b0*(c + dt*R(c))
inline int launch_element(const dg_mesh *m, const double *c, const double *u0, double *out,
                          double *trace_out, const double *fhat, double dt, double a0, double b0,
                          int mode, void *stream) {
  return launch_element(m, c, u0, out, trace_out, fhat, shu_osher(dt, a0, b0), mode, stream);
}
// Mixed-precision element kernel (tcgen05, kind::tf32); split3 selects 3xTF32.
// Work space of the mixed-precision modes, carved from the float64 trace and
// flux buffers: traces float32 [N][3*ne][M]; edge fluxes float32 [F][ne][M]
// followed by their float64 mean-mode integrals [F][M] (fits for ne >= 2).
struct MixedBuffers { float *trace; float *fhat; double *fmean; };
MixedBuffers mixed_buffers(const dg_mesh *m, double *trace, double *fhat);
int launch_face_flux_mixed(const dg_mesh *m, const MixedBuffers &b, void *stream);
// Tensor-core element kernel: as launch_element (mode 0/1) with float32 traces
// and fluxes; mode 2 writes only the traces of c.
int launch_element_tc(const dg_mesh *m, int split3, const double *c, const double *u0, double *out,
                      float *trace_out, const float *fhat, const double *fmean, const StageUpdate &su,
                      int mode, void *stream);
inline int launch_element_tc(const dg_mesh *m, int split3, const double *c, const double *u0, double *out,
                             float *trace_out, const float *fhat, const double *fmean, double dt, double a0,
                             double b0, int mode, void *stream) {
  return launch_element_tc(m, split3, c, u0, out, trace_out, fhat, fmean, shu_osher(dt, a0, b0), mode, stream);
}
// Builds m->tc_img (synchronous; at mesh creation): the tensor-core kernel's B
// operand images for the mesh's p, n_e and volume rule.  cudaError_t as int.
int tc_tables(dg_mesh *m);
int tc_tables_sym(dg_mesh *m);
// launch_element_tc for a mesh on the symmetric volume rule (dg_mixed_sym.cu)
int launch_element_tc_sym(const dg_mesh *m, int split3, const double *c, const double *u0, double *out,
                          float *trace_out, const float *fhat, const double *fmean, const StageUpdate &su,
                          int mode, void *stream);
int launch_convert_check(int n, unsigned long long *bad, void *stream);
// The fused small-mesh stepper (float64; the limiter a phase of it when on):
// nsteps steps of `method` on c in one cooperative launch, the traces of c
// already in m->trace.  Returns a
// cudaError_t cast to int.  small_rk_fits: whether the mesh is small enough (its
// element tiles fit in one wave of the GPU).
bool small_rk_fits(const dg_mesh *m);
int launch_rk_small(dg_mesh *m, double *c, double dt, int nsteps, int method, void *stream);
int launch_project(const dg_mesh *m, const double *u, double *c, void *stream);
int launch_volume_points(const dg_mesh *m, double *xy, void *stream);
int launch_eval_points(const dg_mesh *m, const double *c, const double *tab, int npts, double *out, void *stream);
int launch_totals(const dg_mesh *m, const double *c, double *out_dev, void *stream);
// det J per element -> out [N]; physical points of npts reference points (rs =
// [npts][2], device) -> out [N][npts][2]; the L2 error of variable var against
// exact [N][npts][4] on the rule (tab [npts][np] basis values, w [npts] weights,
// device) through nb block partials -> out_dev[0]
int launch_det_j(const dg_mesh *m, double *out, void *stream);
int launch_map_points(const dg_mesh *m, const double *rs, int npts, double *out, void *stream);
int launch_l2_error(const dg_mesh *m, const double *c, const double *exact, const double *tab, const double *w,
                    int npts, int var, double *partial, int nb, double *out_dev, void *stream);
// Barth-Jespersen limiter (p = 1) in place on c.  have_traces: trace holds the
// traces of c on entry and holds those of the limited state on return; else the
// traces of the limited state go to trace when it is not null.
int launch_limit(const dg_mesh *m, double *c, double *trace, int have_traces, void *stream);
// largest |v| + c over the volume points -> out_dev[0]
int launch_wave_speed(const dg_mesh *m, const double *c, double *out_dev, void *stream);
// (dR/du)^T lam combined as out = x0 X + x1 Y + x2 Z + s (dR/du)^T lam (X, Y, Z may
// be null).  uvol [N][M][np], G, T, TB [N][3 ne][M] are work buffers.
int launch_rhs_vjp(const dg_mesh *m, const double *u, const double *lam, double *uvol, double *G, double *T,
                   double *TB, const double *X, const double *Y, const double *Z, double x0, double x1,
                   double x2, double s, double *out, void *stream);
// Records a failure message for dg_last_error() and returns st.
dg_status set_error(dg_status st, const char *fmt, ...);
// FMA-rate probe: runs `iters` iterations of 8 independent FMA chains per thread.
int launch_fma_probe(int fp64, int blocks, int threads, int iters, double *out, void *stream);

}  // namespace dg
