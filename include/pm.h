/*
 * pm.h -- C ABI of libpm: the two-species (CDM + neutrino) particle-mesh
 * force step of Emberson et al., "Cosmological neutrino simulations at
 * extreme scale" (CUBEP3M / TianNu), on one NVIDIA GB300 (sm_103a).
 *
 * The step, per the paper:
 *   decompress  the cell-ordered phase-space codes of Sec. 2.4;
 *   deposit     CIC density of both species, each with its own mass, on the
 *               coarse mesh and the buffered fine tiles (Sec. 2.1 footnote,
 *               Sec. 2.3 "density_interpolation", Fig. 1);
 *   solve       forward FFT, Green's-function multiply, three inverse FFTs
 *               (Eqs. 1-3), long range on the coarse mesh and short range
 *               per fine tile (Sec. 2.1);
 *   interpolate CIC force readback (Sec. 2.3 "inverse_force_interpolation");
 *   kick-drift  v' = v + c_kick a, x' = x + c_drift v' (periodic);
 *   recompress  back to the Sec. 2.4 codes with a fresh v_max.
 *
 * Conventions (every entry point):
 *   - positions are float32 in fine-cell units on [0, n_fine), periodic;
 *     velocities float32 in fine cells per unit time; particle arrays are
 *     [n][3] (x, y, z interleaved);
 *   - meshes are dense float32 (or int64 fixed point) arrays indexed
 *     [z][y][x], x fastest; acceleration meshes are [3][z][y][x];
 *   - every pointer argument marked "device" is CUDA device memory owned by
 *     the caller (e.g. a torch tensor's data_ptr()); the library never frees
 *     it.  The library owns its handle, plans, precomputed kernels and
 *     workspace;
 *   - calls are asynchronous and ordered on the given CUDA stream
 *     (cudaStream_t passed as void*; NULL = legacy default stream).  Errors
 *     found while launching are returned; errors found on the device (a
 *     corrupt stream, a capacity overflow) set a sticky status word that
 *     pm_check() returns;
 *   - sizes and indices are 64-bit.
 * Return value of every int function: PM_OK or one PM_ERR_* code; the text
 * of the last error is available from pm_last_error().
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_OK 0
#define PM_ERR_ARG 1      /* null pointer, bad species index, size mismatch */
#define PM_ERR_CONFIG 2   /* unsupported configuration in pm_init */
#define PM_ERR_CUDA 3     /* a CUDA runtime call failed */
#define PM_ERR_CORRUPT 4  /* compressed stream fails validation */
#define PM_ERR_OVERFLOW 5 /* a caller-sized capacity (escape list) was exceeded */
#define PM_ERR_RANGE 6    /* position outside [0, n_fine) handed to the codec */
#define PM_ERR_TIMEOUT 7  /* a bounded device wait gave up */

typedef struct pm_handle pm_handle_t;

/* Problem statement (Sec. 2.1): meshes, tiles, species and the split.
 * Lengths are fine-mesh cells throughout, so the box is n_fine cells on a
 * side and there is no separate box length: a caller with a box of side L
 * passes positions x n_fine / L, velocities v n_fine / L (per unit of the
 * time variable of c_kick and c_drift) and G (n_fine / L)^3 (mass units
 * unchanged), and scales the results back.
 *  n_fine        fine-mesh cells per side; positions live on [0, n_fine).
 *  coarse_ratio  fine cells per coarse cell (the paper uses 4: the short-
 *                range mesh is 4x finer than the long-range one).  1 selects
 *                a single periodic mesh solved with the full Green's
 *                function of Eq. 2 (no tiles, no split); its edge n_fine
 *                must be one of 16, 32, 48, 64, 96, 128.  In two-level mode
 *                the coarse edge n_fine / coarse_ratio must be one of those
 *                or 192, 256, 384 (n_fine up to 1536).
 *  tile, buffer  fine-tile interior edge t and buffer width b (Fig. 1);
 *                tile edge T = t + 2b must be one of 16, 32, 48, 64, 96,
 *                128; t must divide n_fine; T <= n_fine.
 *  cmp_ratio     fine cells per compression ("linked-list") cell (Sec. 2.4
 *                bins on the coarse mesh: 4); a power of two.  In two-level
 *                mode it must equal coarse_ratio.
 *  vel_bits      16 (the paper's 2-byte velocities) or 8 (reduced precision).
 *  deposit_mode  0: float32 CIC with atomics (the fused step bins each cell
 *                block in 32-bit fixed point, scaled per block so that no
 *                cell overflows, and adds the block to the float32 mesh);
 *                1: int64 fixed point (mass in
 *                units of 2^-32, conservative integer split) -- bit-exact and
 *                independent of particle order.
 *  G             gravitational constant in these units.
 *  mass, count   per species (0 = CDM, 1 = neutrinos).
 *  r_split       Gaussian split scale r_s in fine cells (two-level).
 *  r_cut         short-range kernel radius R in fine cells, R <= b - 2.
 *  tile_batch    fine tiles solved per batch (0 = library default).
 *  vmax_mode     v_max' of the recompressed velocities (Sec. 2.4): 0 = the
 *                exact max over particles and components of |v'_d| (the
 *                paper's definition; needs the whole kicked population before
 *                any velocity can be quantised); 1 = the bound
 *                v_max + |c_kick| (max|a_coarse| + max|a_fine|) over the
 *                force meshes, rounded up, known right after the solve, so
 *                pm_step quantises velocities in the same pass that kicks
 *                them.  Mode 1 is not the paper's definition: the codes
 *                differ from mode 0 (coarser velocity bins), but every
 *                |v'_d| is still <= v_max'.  With pp = 1 the bound adds
 *                |c_kick| max_i |a_pp,i|.
 *  pp            1: add the particle-particle force of Eq. 4 (direct sum over
 *                the particles sharing a fine-mesh cell [i, i+1)^3, both
 *                species, pairs closer than r_soft dropped) to every
 *                particle's acceleration in pm_step; 0: PM force only.
 *  r_soft        PP softening length in fine cells (Sec. 2.1: 0.05 of the
 *                mean inter-particle spacing); used when pp = 1. */
typedef struct pm_config {
  int32_t n_fine;
  int32_t coarse_ratio;
  int32_t tile;
  int32_t buffer;
  int32_t cmp_ratio;
  int32_t vel_bits;
  int32_t deposit_mode;
  int32_t tile_batch;
  int32_t vmax_mode;
  int32_t pp;
  double G;
  double mass[2];
  int64_t count[2];
  double r_split;
  double r_cut;
  double r_soft;
} pm_config_t;

/* One species' compressed state (Sec. 2.4) in device memory, SoA layout:
 *  n        particle count (host value; particles are conserved by a step).
 *  cnt      [n_cmp^3] count byte per compression cell, cells ordered
 *           c = ix + n_cmp (iy + n_cmp iz); 255 = "see escape list".
 *  esc      [esc_cap][2] uint32 pairs (cell, count) for cells holding >= 255
 *           particles, ascending by cell (the paper's 4-byte count).
 *  esc_cap  capacity of esc in pairs (written by compress, read by decompress).
 *  n_esc    device uint32: number of valid pairs in esc.
 *  pos      [n][4] uint8: in-cell offsets (px, py, pz) = floor(256 * offset /
 *           cell width), then one zero pad byte (a 4-byte word per particle).
 *  vel      [n][4] uint16 (vel_bits 16) or uint8 (vel_bits 8): (vx, vy, vz,
 *           0) with v_d -> floor(v_d 2^(b-1) / v_max + 2^(b-1)) clamped to
 *           [0, 2^b - 1].  The pad makes every particle's codes one aligned
 *           word each (8 or 12 bytes in memory); the serialized stream of
 *           pm_serialize carries no pads (9 or 6 bytes per particle).
 *  vmax     device float32: v_max of this species, max over particles and
 *           components of |v_d| (the paper's per-species header value).
 * Particles are stored cell by cell in cell order; within a cell the order
 * is unspecified (the paper leaves it open). */
typedef struct pm_codes {
  int64_t n;
  uint8_t* cnt;
  uint32_t* esc;
  int64_t esc_cap;
  uint32_t* n_esc;
  uint8_t* pos;
  void* vel;
  float* vmax;
} pm_codes_t;

/* Uncompressed particles of one species in device memory: x, v [n][3]. */
typedef struct pm_particles {
  int64_t n;
  float* x;
  float* v;
} pm_particles_t;

/* Host-memory twin of pm_codes_t for pm_step_host and the serializer: same
 * fields and layouts, every pointer is host memory (pinned for speed). */
typedef pm_codes_t pm_host_codes_t;

/* Validates cfg, allocates the workspace and precomputes, in float64 on the
 * host then rounded to float32, the coarse Green's function (Eq. 2 with the
 * Gaussian long-range factor, or the full Eq. 2 for a single mesh) and the
 * DFT of the short-range tile kernel.  Uses the current CUDA device; blocks
 * until the tables are uploaded.  *out receives the handle.
 * Errors: PM_ERR_ARG (null), PM_ERR_CONFIG (see pm_config_t), PM_ERR_CUDA. */
int pm_init(const pm_config_t* cfg, pm_handle_t** out);

/* Frees the handle and its workspace (synchronises its device first). */
int pm_destroy(pm_handle_t* h);

/* Sizes derived from the config (host values): compression cells per side,
 * coarse cells per side (0 for a single mesh), fine tiles, tile edge T. */
int pm_geometry(const pm_handle_t* h, int64_t* n_cmp, int64_t* n_coarse, int64_t* n_tiles,
                int64_t* tile_edge);

/* Decompress one species (Sec. 2.4): x, v device [n][3] float32, in stream
 * (cell) order.  Positions decode at bin centres:
 *   x_d = (c_d + (q_d + 1/2) / 256) * cmp_ratio,
 *   v_d = ((q_d - 2^(b-1)) + 1/2) * v_max / 2^(b-1).
 * Validation (count bytes vs escape list vs in->n, v_max finite >= 0)
 * reports PM_ERR_CORRUPT through pm_check(). */
int pm_decompress(pm_handle_t* h, int species, const pm_codes_t* in, float* x, float* v, void* stream);

/* pm_decompress for callers that cannot allocate device memory.  The paper
 * has no counterpart: this exists for embedding applications that own the
 * whole device memory budget and forbid libraries to allocate, and for host
 * threads that must not pay the device-wide synchronisation cudaMalloc and
 * cudaFree can cause.  No handle is needed and nothing is allocated: the
 * scratch (CSR offsets of at most 64^3 compression cells, scan partials and a
 * status word, about 2.1 MB) is one fixed __device__ array inside the library,
 * which every GPU that loads the library keeps until the process exits.
 *  n_fine, cmp_ratio, vel_bits  as in pm_config_t; (n_fine/cmp_ratio)^3 must
 *                               not exceed 64^3, else PM_ERR_ARG;
 *  in, x, v                     as in pm_decompress (device memory, caller-owned).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * process; make that first call before any stream capture starts.  The
 * address belongs to the device's primary context: after cudaDeviceReset it
 * is stale, so do not call this entry point again on a device that has been
 * reset.  Every call shares the one array and
 * leaves its contents behind; calls that overlap on the GPU (other streams,
 * other host threads) race on it, so the caller must serialise them.  The
 * call synchronises `stream` before returning and reports a corrupt stream
 * as PM_ERR_CORRUPT directly (there is no handle to query). */
int pm_decompress_noalloc(int32_t n_fine, int32_t cmp_ratio, int32_t vel_bits, const pm_codes_t* in, float* x,
                          float* v, void* stream);

/* Compress one species (Sec. 2.4) from device float32 x, v [in->n][3] (x in
 * [0, n_fine)).  v_max is the exact max |v_d| unless vmax_in (device float)
 * is given.  out->cnt/esc/n_esc/pos/vel/vmax are written; out->n must equal
 * the particle count.  Escape-list overflow -> PM_ERR_OVERFLOW (pm_check);
 * a position outside [0, n_fine) -> PM_ERR_RANGE (pm_check). */
int pm_compress(pm_handle_t* h, int species, const float* x, const float* v, const float* vmax_in,
                pm_codes_t* out, void* stream);

/* CIC deposit (Sec. 2.3) of n particles of one species, mass cfg.mass[s],
 * ADDED into the caller's meshes (zero them first): rho_fine [n_fine^3],
 * rho_coarse [n_coarse^3] (two-level only, else NULL).  Fine tiles are
 * periodic windows of rho_fine: tile (i,j,k) covers fine cells
 * (i t - b .. i t + t + b - 1, ...) mod n_fine (see pm_tile_density). */
int pm_deposit(pm_handle_t* h, int species, const float* x, int64_t n, float* rho_coarse,
               float* rho_fine, void* stream);

/* CIC deposit of per-particle weights onto the fine mesh (the convention of
 * pm_deposit, periodic): w [n][nw] float32 (1 <= nw <= 4) on device, out
 * [nw][n_fine^3] float32, ADDED to.  The compression study of Sec. 2.4
 * measures number and momentum densities with it (weights 1, v_x, v_y, v_z).
 * x [n][3] in fine cells, [0, n_fine).  PM_ERR_ARG for nw outside 1..4. */
int pm_deposit_weights(pm_handle_t* h, const float* x, int64_t n, const float* w, int32_t nw, float* out,
                       void* stream);

/* Same, int64 fixed point: each particle's mass llrint(m 2^32) is split
 * exactly over its 8 CIC corners, one dimension at a time, with weights
 * floor(f 2^20) (f = x - floor(x) in float32).  Bit-exact, order-free. */
int pm_deposit_fixed(pm_handle_t* h, int species, const float* x, int64_t n, int64_t* rho_coarse,
                     int64_t* rho_fine, void* stream);

/* The fused deposit that pm_step runs: decodes both species' positions from
 * their codes and deposits them (masses cfg.mass) into the caller's meshes,
 * binned in shared memory per block of compression cells.  Meshes are
 * float32, or int64 when cfg.deposit_mode == 1; they are ADDED to.
 * Validation of the codes as in pm_decompress. */
int pm_deposit_codes(pm_handle_t* h, const pm_codes_t in[2], void* rho_coarse, void* rho_fine, void* stream);

/* Copies fine tile `tile` (index ix + nt (iy + nt iz)) of the periodic fine
 * density into out [T^3]: the window the tile solve transforms.  On cells
 * 1..T-2 it equals a CIC deposit of exactly the particles whose stencil lies
 * inside the tile. */
int pm_tile_density(pm_handle_t* h, const float* rho_fine, int64_t tile, float* out, void* stream);

/* Solve (Eqs. 1-3, Sec. 2.1).  Single mesh: acc_fine [3][n_fine^3] =
 * acceleration at the fine mesh points, acc_coarse unused.  Two level:
 * acc_coarse [3][n_coarse^3] long-range acceleration on the coarse mesh;
 * acc_fine [3][n_fine^3] short-range acceleration, each tile contributing its
 * interior t^3 cells.  rho_* as produced by pm_deposit (float32 mode). */
int pm_solve(pm_handle_t* h, const float* rho_coarse, const float* rho_fine, float* acc_coarse,
             float* acc_fine, void* stream);

/* Same, reading int64 fixed-point densities (mass units 2^-32). */
int pm_solve_fixed(pm_handle_t* h, const int64_t* rho_coarse, const int64_t* rho_fine, float* acc_coarse,
                   float* acc_fine, void* stream);

/* CIC force interpolation: a [n][3] = coarse CIC gather (positions /
 * coarse_ratio) + fine CIC gather, at device positions x [n][3]. */
int pm_interpolate(pm_handle_t* h, const float* x, int64_t n, const float* acc_coarse,
                   const float* acc_fine, float* a, void* stream);

/* Interpolate, then kick and drift in place: v' = v + c_kick a,
 * x' = x + c_drift v' wrapped into [0, n_fine). */
int pm_kick_drift(pm_handle_t* h, float* x, float* v, int64_t n, const float* acc_coarse,
                  const float* acc_fine, double c_kick, double c_drift, void* stream);

/* One fused PM step from compressed state to compressed state for both
 * species: decompress + deposit, solve, interpolate + kick + drift +
 * recompress, with the library's own meshes and per-particle scratch (sized
 * at pm_init for count[0] + count[1] particles; larger inputs return
 * PM_ERR_ARG).  in[s] and out[s] must not alias; out[s].n must equal
 * in[s].n.  v_max of the output is the exact per-species max |v'_d|.
 * Within a cell the output order is unspecified. */
int pm_step(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift,
            void* stream);

/* pm_step from HOST buffers: copies both species' codes host -> device,
 * steps, copies the result codes device -> host, on `stream`, and
 * synchronises it before returning.  Device staging buffers are owned by
 * the handle (allocated on first use).  Returns the device status too. */
int pm_step_host(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                 double c_drift, void* stream);

/* Packed codes: the same pm_codes_t fields, but pos points to u8[n][3]
 * (px, py, pz) and vel to u8[n][3] or u16[n][3] (vx, vy, vz, little-endian):
 * the Sec. 2.4 record bytes without the one-word-per-particle padding of the
 * in-memory form (6 or 9 bytes per particle instead of 8 or 12).
 * pm_pack_codes / pm_unpack_codes convert between the forms in device memory
 * (cnt, esc, n_esc and vmax are copied as they are); padded pos/vel must be
 * 16-byte aligned, packed pos 4-byte and packed vel 4-byte (8-bit) or 8-byte
 * (16-bit) aligned, out->n == in->n and out->esc_cap >= in->esc_cap.
 * pm_step_packed is pm_step_host with packed host codes: only the record
 * bytes cross the host link, and the library (un)packs them on the device.
 * The paper keeps its compressed particles in this record form. */
int pm_pack_codes(pm_handle_t* h, const pm_codes_t* in, pm_codes_t* out, void* stream);
int pm_unpack_codes(pm_handle_t* h, const pm_codes_t* in, pm_codes_t* out, void* stream);
int pm_step_packed(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                   double c_drift, void* stream);

/* pm_step_packed without waiting: queues the input copies (host -> device
 * on a library stream, then unpacked there), the step on `stream`, and the
 * output copies (device -> host on a second library stream), and returns.
 * Consecutive calls overlap: a call's position records go into the library's
 * packed staging once the previous call has unpacked its own (beside the
 * previous step), are unpacked once the previous step has read its input
 * (after its count pass), and its velocity records follow (beside the
 * previous scatter and this call's deposit and solve); one step's output
 * copies run beside the next step's input copies, deposit, solve and (when
 * the device has room for a packed output buffer of its own, 9 or 6 bytes
 * per particle, with 2 GB to spare) its count pass and scatter; without that
 * room the packed output shares the step scratch and the next count pass
 * waits for the copies.  `out` is complete,
 * and `in` may be changed, only after pm_check (which synchronises `stream`
 * and both library streams and reports the status); the host buffers must
 * stay valid until then, and a caller that reuses one `out` for several
 * calls keeps the last step's codes.  Needs device memory for one more
 * packed copy of the input (9 or 6 bytes per particle) beyond
 * pm_step_packed's, allocated on the first call.  Graph replay does not
 * apply to this call. */
int pm_step_packed_async(pm_handle_t* h, const pm_host_codes_t in[2], pm_host_codes_t out[2], double c_kick,
                         double c_drift, void* stream);

/* Reverse mode of the single-mesh step (coarse_ratio == 1), for gradients of
 * losses of the final positions or density with respect to initial
 * conditions.  The paper has no adjoint; these are the chain rule of the
 * forward step above (Sec. 2.1 Eqs. 1-3, Sec. 2.3 CIC, kick-drift).  Two-level
 * handles return PM_ERR_CONFIG.
 *
 * pm_deposit_adjoint:     lam_x[p] += m_s sum_c lam_rho(c) grad_x W(x_p - c)
 *                          (W = CIC weight; lam_rho [n_fine^3] float32).
 * pm_solve_adjoint:       lam_rho = A^T lam_acc for a = A rho of pm_solve
 *                          (kernel conj(i k_d g)); lam_acc [3][n_fine^3].
 * pm_interpolate_adjoint: the reverse of interpolate + kick + drift for one
 *                          species: lam_v += c_drift lam_x; lam_a = c_kick lam_v;
 *                          lam_acc(c) += lam_a W(x - c) (atomics, zero it
 *                          first); lam_x += sum_c (lam_a . acc(c)) grad W.
 * pm_step_adjoint:        one whole reverse step for both species: recomputes
 *                          the step's acceleration at the pre-step positions
 *                          state[s].x (cfg.deposit_mode as in the forward; use
 *                          the fixed-point mode for a bit-exact recompute), then
 *                          maps lam[s] = (dL/dx', dL/dv') after the step to
 *                          (dL/dx, dL/dv) before it, in place.
 * pm_step_adjoint_acc:    the same reverse step with the step's acceleration
 *                          mesh supplied (acc_fine [3][n^3] float32, device,
 *                          read only: pm_solve's output at the pre-step
 *                          positions, e.g. kept from a checkpoint segment's
 *                          recompute), so nothing is recomputed.  PM_ERR_ARG
 *                          for a null mesh. */
int pm_deposit_adjoint(pm_handle_t* h, int species, const float* x, int64_t n, const float* lam_rho, float* lam_x,
                       void* stream);
int pm_solve_adjoint(pm_handle_t* h, const float* lam_acc, float* lam_rho, void* stream);
int pm_interpolate_adjoint(pm_handle_t* h, const float* x, int64_t n, const float* acc_fine, double c_kick,
                           double c_drift, float* lam_x, float* lam_v, float* lam_acc, void* stream);
int pm_step_adjoint(pm_handle_t* h, const pm_particles_t state[2], pm_particles_t lam[2], double c_kick,
                    double c_drift, void* stream);
int pm_step_adjoint_acc(pm_handle_t* h, const pm_particles_t state[2], pm_particles_t lam[2], const float* acc_fine,
                        double c_kick, double c_drift, void* stream);

/* Synchronises `stream`, returns and clears the sticky device status
 * (PM_OK, PM_ERR_CORRUPT, PM_ERR_OVERFLOW, PM_ERR_RANGE, PM_ERR_TIMEOUT). */
int pm_check(pm_handle_t* h, void* stream);

/* Diagnostic of the bounded device waits (the mbarrier waits of the
 * TMA-staged tile solve, which give up after about a second and record a
 * timeout instead of hanging): launches on `stream` one block that waits on
 * an mbarrier phase no copy ever completes, gives up after limit_cycles SM
 * clock cycles (1e3 .. 2e9, else PM_ERR_ARG) and records the timeout in the
 * handle's status word, so the next pm_check returns PM_ERR_TIMEOUT (and
 * clears the word).  No copy is in flight when the block exits, and the
 * handle stays usable. */
int pm_wait_probe(pm_handle_t* h, int64_t limit_cycles, void* stream);

/* Copies the last error message (NUL-terminated, truncated to n). */
int pm_last_error(const pm_handle_t* h, char* buf, size_t n);

/* Coarse density from a fine one (two-level handles): rho_coarse[C] =
 * sum_k w(kx) w(ky) w(kz) rho_fine[rc C + k], w(k) = 1 - |k|/rc for
 * |k| < rc (periodic; rc = coarse_ratio).  For CIC this equals depositing
 * the particles on the coarse mesh directly (the coarse tent is piecewise
 * linear on fine nodes), so the float pm_step deposits only the fine mesh
 * and restricts it; likewise it adds the coarse force, trilinearly
 * interpolated onto the fine nodes, to the fine force mesh and interpolates
 * the particles from that one mesh.  float32 [nc^3] / [n^3], overwritten.
 * No counterpart in the paper. */
int pm_restrict(pm_handle_t* h, const float* rho_fine, float* rho_coarse, void* stream);

/* Particle-particle acceleration of Eq. 4 (Sec. 2.1) for every particle of
 * the compressed state in[2]: a_i = G sum m_j (x_j - x_i)/|x_j - x_i|^3 over
 * the particles of both species in particle i's fine-mesh cell, pairs closer
 * than cfg.r_soft dropped.  acc: device float32 [n0 + n1][4] (16-byte
 * aligned), row t = stream index (species 0 first), components x, y, z, 0.
 * The step adds the same values when cfg.pp = 1. */
int pm_pp_accel(pm_handle_t* h, const pm_codes_t in[2], float* acc, void* stream);

/* Asynchronous checkpoint of a compressed state (the single-GPU analogue of
 * writing checkpoints through a RAM burst buffer): pm_checkpoint_begin
 * queues device -> host copies of both species' codes (cnt, the esc_cap
 * escape pairs, n_esc, pos, vel, vmax; same padded layouts) into the
 * caller's host buffers on a library-owned stream, ordered after the work
 * already queued on `stream`, and returns at once; the caller keeps
 * stepping meanwhile.  The device codes must not be overwritten until the
 * copies are done: pm_checkpoint_fence(h, s) makes stream s wait for them
 * (no host block), pm_checkpoint_wait(h) blocks the host until they are
 * done, after which the host codes hold the state and pm_serialize turns
 * them into the Sec. 2.4 byte stream.  One checkpoint may be pending per
 * handle (PM_ERR_ARG otherwise).  Host buffers should be pinned; host[s].n
 * must equal codes[s].n and host[s].esc_cap >= codes[s].esc_cap. */
int pm_checkpoint_begin(pm_handle_t* h, const pm_codes_t codes[2], pm_host_codes_t host[2], void* stream);
int pm_checkpoint_fence(pm_handle_t* h, void* stream);
int pm_checkpoint_wait(pm_handle_t* h);

/* Per-stage timing of pm_step with CUDA events on its stream: enable (1) or
 * disable (0); pm_stage_times writes up to cap averages in ms over the
 * steps since enabling, names into the ';'-separated buffer. */
int pm_set_timing(pm_handle_t* h, int on);
int pm_stage_times(pm_handle_t* h, float* ms, int cap, int* n_stages, char* names, size_t names_cap);

/* Graph replay of pm_step (and pm_step_host): with on = 1, the first pm_step
 * with a given set of codes descriptors (in[2], out[2], every field) and
 * (c_kick, c_drift) captures its launch sequence into a CUDA graph on a
 * library-owned stream; later calls with the same set launch that graph on
 * the caller's stream.  Up to 8 graphs are kept (oldest evicted), so a
 * ping-pong pair of codes buffers replays two graphs.  The graph holds the
 * device pointers it was captured with: the caller must not free or reuse
 * those buffers for other data while graphs are on (turn them off, or
 * destroy the handle, first).  on = 0 synchronises the device and drops every
 * graph.  Per-stage timing (pm_set_timing) bypasses the graphs.  No
 * counterpart in the paper (launch batching only; results are identical). */
int pm_set_graphs(pm_handle_t* h, int on);

/* Launch tuning of pm_step and pm_deposit_codes (no counterpart in the paper;
 * results are the same for every tuning up to float summation order):
 *  deposit_block[3]    compression cells per deposit CTA along x, y, z (its
 *                      shared-memory bins cover them plus a one-cell halo);
 *  deposit_persistent  0: one CTA per cell block; 1: as many CTAs as fit on
 *                      the device, each drawing cell blocks from a device
 *                      counter until none are left (uneven, clustered blocks
 *                      then balance across the SMs);
 *  kick_block[3]       compression cells per CTA of the interpolate + kick +
 *                      drift + recompress passes;
 *  kick_window         half-width in cells of the new-cell window whose
 *                      counts a CTA keeps in shared memory (1..4; particles
 *                      moving further use global counters);
 *  kick_persistent     as deposit_persistent, for those passes;
 *  tile_batch          fine tiles per solve launch, 1..the configured batch.
 * Every block edge must divide n_cmp and the shared memory must fit one block
 * of the device (PM_ERR_ARG otherwise).  pm_set_tuning drops captured step
 * graphs (synchronising the device first). */
typedef struct pm_tuning {
  int32_t deposit_block[3];
  int32_t deposit_persistent;
  int32_t kick_block[3];
  int32_t kick_window;
  int32_t kick_persistent;
  int32_t tile_batch;
} pm_tuning_t;
int pm_get_tuning(const pm_handle_t* h, pm_tuning_t* t);
int pm_set_tuning(pm_handle_t* h, const pm_tuning_t* t);

/* Autotuner: times pm_step(in -> out, c_kick, c_drift) on `stream` (one
 * warm-up step, then `reps` timed steps per candidate, CUDA events) for the
 * current tuning and for candidate deposit blocks and launch forms, then
 * candidate kick blocks, windows and launch forms, then tile batches
 * (coordinate search, each stage starting from the best so far), keeps the
 * fastest and writes it to *chosen (may be NULL).  It writes `out` (any
 * earlier content is lost) and never `in`; blocks the calling thread until
 * the timing is done.  Per-stage timing and step graphs are suspended while
 * it runs.  On error the previous tuning is restored. */
int pm_autotune(pm_handle_t* h, const pm_codes_t in[2], pm_codes_t out[2], double c_kick, double c_drift, int32_t reps,
                void* stream, pm_tuning_t* chosen);

/* Serializer for the Sec. 2.4 byte stream (host memory, not stream-ordered):
 * header "PMNU", u32 version 1, u32 n_cmp, u32 vel_bits, u64 n, f32 v_max,
 * u32 0; then per cell the count byte (255 + int32 count if >= 255) and the
 * cell's records px py pz (u8) vx vy vz (u16 LE or u8).  `codes` points to
 * host copies (cnt, esc, *n_esc, pos, vel, *vmax).  With buf == NULL only
 * *len is computed. */
int pm_serialize(const pm_host_codes_t* codes, int32_t n_cmp, int32_t vel_bits, uint8_t* buf, size_t cap,
                 size_t* len);
int pm_deserialize(const uint8_t* buf, size_t len, int32_t n_cmp, int32_t vel_bits, pm_host_codes_t* codes);

const char* pm_error_string(int code);

/* Number of CUDA kernels the library has launched in this process (all
 * handles), for launch accounting in benchmarks. */
int64_t pm_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PM_H */
