// internal.h -- declarations shared by the translation units of libfitgb.so.
//
// Device layout.  Every field component and every per-edge/per-face
// coefficient is a "pitched" array of pitch*ny*nz values: x fastest with the
// row padded to pitch = nx rounded up to a multiple of 4, so every row starts
// on a 16-byte boundary (the alignment TMA tensor copies need).  Padding
// entries are zero and stay zero.  The ABI's compact layout (rows of nx) is
// converted at the edges with 2-D copies.
//
// One leapfrog state is one block of 6 components: e_x, e_y, e_z, h_x, h_y,
// h_z.  Each member owns two blocks and the fused step reads one and writes
// the other (ping-pong), so tiles never race on their halos.  All member
// blocks of a run sit in one allocation, block b of member q at index
// 2q + b, so one 5-D tensor map (x, y, z, component, block) covers them all.
//
// Coefficients: one allocation of 3 or 6 components: cb_x, cb_y, cb_z and,
// for lossy grids, ca_x, ca_y, ca_z (so one tensor copy brings both).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "fitgb.h"

namespace fitgb {

constexpr double kPi = 3.14159265358979323846;
constexpr double kC0 = 299792458.0;                  // [m/s]
constexpr double kMu0 = 4.0e-7 * kPi;                // [H/m]
constexpr double kEps0 = 1.0 / (kMu0 * kC0 * kC0);   // [F/m]

constexpr int kMaxSrc = 8;    // sources fused into one step launch
constexpr int kMaxPrb = 32;   // probes fused into one step launch

// Device error word bits.
enum : int { kErrIndex = 1, kErrTimeout = 2 };

inline int pitch_of(int nx) { return (nx + 3) & ~3; }

struct EdgeRef {
    int axis, i, j, k;
};

// One leapfrog member: a state pair plus its place in absolute time.
struct Member {
    void *st[2];            // the two 6-component state blocks (T)
    int blk[2];             // their block indices in the run's state allocation
    long long start;        // absolute step of the member at iteration 0
    long long end;          // absolute step it stops at (batched launches skip it there)
    long long src_lo;       // sources act for absolute steps in [src_lo, src_hi)
    long long src_hi;
    double *probe;          // probe rows, row = absolute step - probe_base
    long long probe_base;
    double *energy;         // energy[absolute step - energy_base]
    long long energy_base;
};

// Arguments of one fused leapfrog launch (all members advance one step).
template <typename T>
struct StepArgs {
    int nx, ny, nz, pitch;
    long long ncell;        // pitch*ny*nz: the stride between components
    int tiles_x, tiles_y, nchunk, kz;
    const T *cb;    // 3 components
    const T *ca;    // 3 components, or null when the grid is lossless (ca = 1)
    const T *ch;    // 3 values (uniform mu) or 3 components (per face)
    const T *meps;  // 3 components, energy only
    const T *mmu;   // 3 values or 3 components, energy only
    const Member *mem;
    int nmem;       // members in this launch (table prefix)
    int it;         // iteration: member m is at absolute step mem[m].start + it
    int parity;     // read st[parity], write st[parity ^ 1]
    const double *amp;      // source amplitudes amp[(step - amp_base)*nsrc + s]
    long long amp_base;
    long long amp_len;
    int nsrc;
    EdgeRef src[kMaxSrc];
    int nprb;
    EdgeRef prb[kMaxPrb];
    int *err;
    int wait_limit;   // polls before an mbarrier wait gives up (0: default)
    int extra_tx;     // test hook: bytes announced beyond a tile's first plane
    // adjoint gradient fused into the step (FP32 TMA kernel; gb null = off):
    // gb_a += gk_a * (mu_a * (e1_a - e0_a)) on every edge of the grid, mu the
    // step's input e (the adjoint state), e1/e0 3 pitched components each
    const T *ge1, *ge0;
    float *gb;
    float gk[3];
    // forward sweep keeping e^{n+1} - e^n for the adjoint (FP32 two-cell TMA kernel; null = off):
    // 3 pitched components; an adjoint step then takes them in ge1 with ge0 null
    float *gd;
    // set: a launch call launches nothing and stores how many CTAs of the kernel it
    // would launch fit on one SM
    int *occ_out;
};

// The occupancy answer of a launch call made with StepArgs::occ_out set.
template <typename K>
inline cudaError_t report_occupancy(K kernel, int threads, size_t dyn_smem, int *out) {
    *out = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, kernel, threads, dyn_smem);
}

// One grid of a batched launch (device table).
template <typename T>
struct GridDesc {
    int nx, ny, nz, pitch;
    long long ncell;          // pitch*ny*nz
    int tiles_x, tiles_y, nchunk, kz;
    const T *ch;              // 3 values or 3 pitched components
    int muarr;
    const Member *mem;        // this grid's member table
    const double *amp;        // this grid's source table
    long long amp_base;
    int nsrc, nprb;
    EdgeRef src[kMaxSrc];
    EdgeRef prb[kMaxPrb];
};

// One unit of work of a batched step: a tile column of one member of one grid.
struct WorkItem {
    int grid, member, tile, chunk;
};

// Arguments of one batched launch (all active members of all grids, one step).
template <typename T>
struct BatchArgs {
    const GridDesc<T> *grids;
    const CUtensorMap *maps;  // 2 per grid (state, coefficients), 64-byte aligned
    const WorkItem *items;
    int nitems;               // items of the launch (inactive members are skipped)
    int it, parity;
    int *counter;             // work counter of this launch (zero before it)
    int *err;
};

struct Tile {
    int tx, ty, kz;
    int kernel;      // 1: shared-memory staging by plain loads, 2: TMA pipeline
    int stages = 0;  // TMA ring depth (0: the tile's default)
    bool single = false;   // FP32 TMA kernels: one cell per thread instead of two
    bool kz_fixed = false; // kz given by the caller (else chosen per run, see chunk_length)
};

// step.cu: plain-load staging kernel
template <typename T>
cudaError_t launch_step(const StepArgs<T> &a, Tile tile, bool lossy, bool mu_array, bool energy,
                        cudaStream_t s);
bool tile_supported(int tx, int ty);

// step_tma.cu: TMA-pipelined kernel
struct TmaMaps {
    CUtensorMap state;   // (x, y, z, component, block), box (tx+8, ty+2, 1, 3, 1)
    CUtensorMap coef;    // (x, y, z, component), box (tx, ty, 1, 3 or 6)
};
template <typename T>
cudaError_t launch_step_tma(const StepArgs<T> &a, const TmaMaps &maps, Tile tile, bool lossy, bool mu_array,
                            bool energy, cudaStream_t s);
bool tma_tile_supported(int tx, int ty, int elem_bytes);
// tiles of the FP32 TMA step kernel with the fused adjoint gradient (StepArgs::gb)
bool step_grad_supported(Tile tile);
// batched persistent kernel (FP32): launch over b.nitems items with `ctas` CTAs
cudaError_t launch_batched_f32(const BatchArgs<float> &b, Tile tile, bool lossy, int ctas, cudaStream_t s);
int batched_ctas_per_sm_f32(Tile tile, bool lossy);
bool batched_tile_supported(int tx, int ty);
// Encode the two tensor maps of a run; returns false if the driver lacks TMA.
// nstate: components per state block (6, or 12 for compensated fields)
bool encode_tma_maps(TmaMaps *out, int elem_bytes, int nx, int ny, int nz, int pitch, void *state,
                     int nblocks, const void *coef, int ncoef, int tx, int ty, int nstate = 6);

// step2_tma.cu: two steps per launch (FP32, no energy); tm_state with the box (tx+8, ty+4, 1, 3, 1),
// tm_coef the coefficient window (tx+8, ty+4, 1, 3 or 6)
bool step2_tile_supported(int tx, int ty);
cudaError_t launch_step2_tma(const StepArgs<float> &a, const CUtensorMap &tm_state, const CUtensorMap &tm_coef,
                             int tx, int ty, bool lossy, bool muarr, cudaStream_t s);

// step_comp.cu: compensated FP32 fields (hi + lo pairs, 12-component state blocks)
cudaError_t launch_step_comp(const StepArgs<float> &a, const TmaMaps &maps, Tile tile, bool lossy, bool mu_array,
                             bool energy, cudaStream_t s);
bool comp_tile_supported(int tx, int ty);

// step_res.cu: FP32 fields with bfloat16 residuals (9-component state blocks: 6 hi floats, then the residual
// words (lo e_x, lo e_y), (lo e_z, lo h_x), (lo h_y, lo h_z))
cudaError_t launch_step_res(const StepArgs<float> &a, const TmaMaps &maps, Tile tile, bool lossy, bool mu_array,
                            bool energy, cudaStream_t s);
bool res_tile_supported(int tx, int ty);
// FP64 compact e, h (either may be null = zero) -> one padded state block, masked to the degrees of freedom
cudaError_t split_res(int nx, int ny, int nz, int pitch, const double *e, const double *h, float *state,
                      cudaStream_t s);
// part 0 (e) or 1 (h) of a state block -> FP64 compact fields
cudaError_t join_res(int nx, int ny, int nz, int pitch, const float *state, int part, double *out, cudaStream_t s);
// acc[t] += part 0 (e) or 1 (h) of a state block, padded layout (3*ncp values)
cudaError_t accumulate_res(long long ncp, const float *state, int part, double *acc, cudaStream_t s);

// aux.cu
struct MaterialFlags {
    int bad_eps, bad_mu, bad_sigma, mu_nonuniform, lossy;
    double eps_mu_min;
};
cudaError_t check_materials(const float *eps, const float *mu, const float *sig, long long ncell,
                            MaterialFlags *flags_host, void *scratch, cudaStream_t s);
template <typename T>
cudaError_t build_coeffs(int nx, int ny, int nz, int pitch, const double d[3], const float *eps, const float *mu,
                         const float *sig, double dt, int scheme, bool mu_array, T *ca, T *cb, T *ch,
                         T *meps, T *mmu, cudaStream_t s, bool round_float = false);
cudaError_t source_table(const fit_source *src_dev, int nsrc, long long base, long long len, double dt,
                         double *amp, cudaStream_t s);
template <typename T>
cudaError_t mask_state(int nx, int ny, int nz, int pitch, T *e, T *h, cudaStream_t s);
template <typename T>
cudaError_t accumulate_state(long long n, const T *st, double *acc, cudaStream_t s);
template <typename T>
cudaError_t accumulate_state_kahan(long long n, const T *st, float *sum, float *comp, cudaStream_t s);
cudaError_t kahan_finish(long long n, const float *sum, const float *comp, double *out, cudaStream_t s);
cudaError_t sum_members(int nmem, long long len, const double *per_member, long long stride, double *out,
                        cudaStream_t s);
// compensated fields: FP64 compact (3 components) <-> pitched hi/lo floats
cudaError_t split_pairs(int nx, int ny, int nz, int pitch, const double *in, float *hi, float *lo, int is_h,
                        cudaStream_t s);
cudaError_t join_pairs(int nx, int ny, int nz, int pitch, const float *hi, const float *lo, double *out,
                       cudaStream_t s);
cudaError_t accumulate_pairs(long long n, const float *hi, const float *lo, double *acc, cudaStream_t s);

// graded.cu: tensor-product graded grids (spc_dev: nx + ny + nz sizes, x then y then z)
template <typename T>
cudaError_t build_coeffs_graded(int nx, int ny, int nz, int pitch, const double *spc_dev, const float *eps,
                                const float *mu, const float *sig, double dt, int scheme, T *ca, T *cb, T *ch,
                                T *meps, T *mmu, cudaStream_t s, bool round_float);
// eq. (cfl) with per-cell sizes, and max |row sum| of A (= ||A||_1); scratch: 16 bytes
cudaError_t graded_cfl_and_bound(int nx, int ny, int nz, const double *spc_dev, const float *eps, const float *mu,
                                 void *scratch, double *cfl, double *rowsum_max, cudaStream_t s);

// expo_plan.cu: host side of the Leja / Taylor propagators
constexpr int kExpoMaxDegree = 120;
// (q, m) for dt/dt_CFL = u; FIT_OK or FIT_ERR_ARG.  Cached per argument set.
int expo_plan(int kind, double u, double tol, int precision, int *q, int *m);
// real pair coefficients of the interpolant of exp(a z): alpha[J], gamma[J], eta2[J], J = m/2
int expo_pair_coeffs(int kind, int m, double a, double *alpha, double *gamma, double *eta2);

// expo.cu: one member of an exponential propagation
template <typename T>
struct ExpoMember {
    T *P;                // accumulator; holds b at a substep's start (6-component pitched block)
    T *R;                // R_{j-1}(X) b
    T *Y;                // X R_{j-1}(X) b
    int nsub;            // substeps of this member
    int blk;             // block index of P in the member blocks (R = blk+1, Y = blk+2) for tensor maps
    const double *fin;   // final substep: [J][4] = alpha_e, gamma_e, alpha_h, gamma_h
    double *basis;       // probe basis: [substep][m+1][nprb] (e at the probe edges)
};

enum ExpoMode { kExpoInit = 0, kExpoPair1 = 1, kExpoPair2 = 2, kExpoSync = 3 };

template <typename T>
struct ExpoArgs {
    int nx, ny, nz, pitch;
    long long ncp;          // padded component stride
    int kz, nchunk;         // z planes per block, chunks along z
    const T *cb;            // 3 components (zero off the degrees of freedom)
    const T *ch;            // 3 values (uniform mu) or 3 components
    double kappa;           // dt_CFL / dt
    const ExpoMember<T> *mem;
    int nmem;               // active members (table prefix)
    int mode;               // ExpoMode
    int pair;               // j = 1..J (pair launches)
    int substep;
    const double *reg;      // [J][2] = alpha, gamma at tau = 1
    double eta2;            // eta_j^2 (second pair launch)
    double sync;            // dt/(2 dt_CFL): half magnetic step in units of X
    int m1;                 // m + 1 (probe basis rows per substep)
    int *err;               // device error word (bounded waits of the TMA pair kernel)
    int extra_tx;           // test hook: bytes announced beyond a tile's first plane (TMA pair kernel)
    int nprb;
    EdgeRef prb[kMaxPrb];
};

template <typename T>
cudaError_t launch_expo(const ExpoArgs<T> &a, bool mu_array, cudaStream_t s);
// probe rows of the Newton basis after an init or a first pair launch
template <typename T>
cudaError_t launch_expo_gather(const ExpoArgs<T> &a, cudaStream_t s);
// dense output: out[m*ostride + (row0[m] + r)*nprb + p] = sum_k D[(r % q)*m1 + k] basis_m[(r/q)*m1 + k][p]
// for r < nrem[m]
cudaError_t launch_expo_dense(int nmem, const double *const *basis, const long long *nrem, const long long *row0,
                              long long max_rows, int q, int m1, int nprb, const double *D, double *out,
                              long long ostride, cudaStream_t s);
// expo_tma.cu: fused pair (y = X r, r' = X y + eta^2 r, p += alpha r + gamma y) with a TMA ring.
// Odd pairs read R and write Y, even pairs the reverse; tm_r covers the member blocks with the
// leapfrog state box (TX+8, TY+2, 1, 3, 1), tm_cb the cb array with the box (TX+8, TY+2, 1, 3).
template <typename T>
cudaError_t launch_expo_pair_tma(const ExpoArgs<T> &a, const CUtensorMap &tm_r, const CUtensorMap &tm_cb,
                                 bool last, bool mu_array, int wait_limit, cudaStream_t s);
// probe rows 2j-1 (r) and 2j (y = X r, computed at the probe edges) of a fused pair
template <typename T>
cudaError_t launch_expo_gather_fused(const ExpoArgs<T> &a, cudaStream_t s);
int expo_pair_tile_x(int elem_bytes);
int expo_pair_tile_y(int elem_bytes);
// a 4-D (x, y, z, component) map over `ncomp` pitched components with an arbitrary box
bool encode_window_map(CUtensorMap *out, int elem_bytes, int nx, int ny, int nz, int pitch, const void *ptr,
                       int ncomp, int box_x, int box_y, int box_c);

// out[t] += sum_m pm[m*stride + t], members in order
cudaError_t add_members(int nmem, long long len, const double *pm, long long stride, double *out, cudaStream_t s);

// adjoint.cu (plen: host array of each probe edge's length)
template <typename T>
cudaError_t adjoint_init(const fit_probe *prb, int nprb, const double *plen, const double *probe_last, const T *cb,
                         T *mu, int pitch, int ny, long long ncp, cudaStream_t s);
cudaError_t adjoint_sources(const fit_probe *prb, int nprb, const double *plen, const double *probe, long long N,
                            double *amp, cudaStream_t s);
template <typename T>
cudaError_t grad_accumulate(long long ncp, const T *mu, const T *e1, const T *e0, const double k[3], double *g,
                            cudaStream_t s);
// FP32 fields: g_b += K mu (e1 - e0) in an FP32 block sum, added into the FP64 total by grad_flush
cudaError_t grad_accumulate_block(long long ncp, const float *mu, const float *e1, const float *e0, const double k[3],
                                  float *gb, cudaStream_t s);
cudaError_t grad_flush(long long ncp, float *gb, double *g, cudaStream_t s);
// spc: device dx[nx], dy[ny], dz[nz] of a graded grid, or null
cudaError_t grad_scatter(int nx, int ny, int nz, int pitch, long long ncp, const double *g, const double *spc,
                         double *grad, cudaStream_t s);
cudaError_t probe_functional(const fit_probe *prb, int nprb, const double *plen, const double *probe, long long N,
                             double *J, cudaStream_t s);

}  // namespace fitgb
