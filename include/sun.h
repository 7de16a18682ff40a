/*
 * sun.h -- C ABI of the GB300 (sm_103a) SU(Nc) pure-gauge link-sweep library.
 *
 * The operations follow Cardoso & Bicudo, "Generating SU(Nc) pure gauge lattice
 * QCD configurations on GPUs with CUDA" (arXiv:1112.4533):
 *   Sec. 2, Eqs. 3-4    Wilson action and plaquette
 *   Sec. 2, Eq. 9       six-plaquette staple
 *   Sec. 2, Eqs. 10-15  SU(2) heatbath and the Cabibbo-Marinari pseudo-heatbath
 *   Sec. 2, Eq. 17      overrelaxation
 *   Sec. 2 (end)        re-unitarization
 *   Sec. 3              hot/cold start, the chessboard (direction x even/odd)
 *                       schedule of eight passes per step, 12-real SU(3) storage
 *
 * Conventions shared by every entry point
 *  - Every call returns a sun_status and never aborts the process.  On failure
 *    sun_last_error() returns a message for the calling thread.
 *  - Lattice extents dims = {Nx, Ny, Nz, Nt} (mu = 0,1,2,3 = x,y,z,t), periodic,
 *    each even and >= 2 (the even/odd colouring must close over the boundary),
 *    and 4*Nx*Ny*Nz*Nt < 2^32 (links are numbered with 32 bits for the RNG).
 *  - Canonical link order (host interchange format, FP64, independent of the
 *    storage format and precision): double[ ((mu*V + lex)*Nc + row)*Nc + col ][2]
 *    with lex = x + Nx*(y + Ny*(z + Nz*t)), V = Nx*Ny*Nz*Nt; i.e. 8*Nc*Nc*V doubles.
 *  - Device work is enqueued on the lattice's CUDA stream and is asynchronous
 *    unless stated otherwise ("syncs").  Host pointers passed in may be pageable
 *    or pinned.
 *  - Random numbers: Philox4x32-10 keyed by the 64-bit seed, counter =
 *    (mu*V + lex, heatbath step, (subgroup << 16) | attempt, 1).  (seed, heatbath
 *    step) is the whole random state of a lattice.
 */
#ifndef SUN_H
#define SUN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SUN_ABI_VERSION 1

typedef struct sun_lattice sun_lattice; /* opaque, owned by the library */

typedef enum {
  SUN_OK = 0,
  SUN_ERR_ARG = 1,         /* an argument is out of range or inconsistent           */
  SUN_ERR_OOM = 2,         /* device memory unavailable or caller buffer too small  */
  SUN_ERR_CUDA = 3,        /* a CUDA runtime call failed                            */
  SUN_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                    */
  SUN_ERR_UNSUPPORTED = 5, /* (Nc, storage, precision) combination not built        */
  SUN_ERR_STATE = 6        /* call not valid in the object's current state          */
} sun_status;

/* update modes of sun_update_pass */
enum { SUN_HEATBATH = 0, SUN_OVERRELAX = 1 };

/*
 * Options of a lattice.  Call sun_options_init() first, then change fields.
 *  precision     32 or 64: link storage and update arithmetic (default 32).
 *                Re-unitarization and the accumulation of the plaquette and the
 *                Polyakov loop are FP64 in both cases.
 *  storage       reals stored per link; 0 picks the default.  Nc=2: 4 (a0..a3 of
 *                Eq. 6, default) or 8 (full 2x2).  Nc=3: 12 (two rows, third row
 *                rebuilt as conj(row0 x row1), Sec. 3, default) or 18 (full).
 *                Nc>=4: 2*Nc*Nc.
 *  reunit_every  sun_sweep re-unitarizes after every reunit_every-th sweep; 0 = never
 *                (default 1).
 *  block_threads CUDA block size of the update passes, 0 = default (128).
 *  stream        cudaStream_t the lattice enqueues on; NULL = a stream the library
 *                creates and owns.
 *  device_buf    optional caller-owned device memory of device_buf_bytes bytes
 *                (>= sun_footprint_bytes) holding all device state of the lattice;
 *                it must be 256-byte aligned and outlive the lattice.  NULL = the
 *                library allocates (cudaMalloc) and frees.
 *  use_graphs    sun_run captures one sweep as a CUDA graph and replays it (default 1).
 *  variant       update-pass kernel variant, bit flags (default 0); results do not
 *                depend on bits 1 and 4:
 *                1 = (SU(3), SU(4) FP32) bound the registers for 5 (SU(3)) or 4
 *                (SU(4), per-link kernel) resident 128-thread blocks per SM;
 *                2 = (SU(3) FP32 two-row storage) multiply out rows 0 and 1 of each
 *                staple term only and take its third row as conj(row0 x row1),
 *                exact for SU(3) products (results move by the order of the
 *                links' unitarity drift, ~1e-6 between re-unitarizations);
 *                4 = (Nc = 4, 6) swap the pass kernel: by default Nc = 6 runs the
 *                row-parallel kernel (Nc threads per link) and Nc = 4 one thread
 *                per link;
 *                8 = run the even and the odd pass of each direction as one
 *                launch, a wavefront over t-slices: odd links of slice t are
 *                updated once the even links of slices t-1, t, t+1 are done
 *                (bitwise the same links as the two passes; the neighbour links
 *                the two parities share are re-read from L2, not HBM).  Kernels
 *                without this form (row-parallel, bit 2) run the two passes.
 *                The device-side waits are bounded: one that gives up after
 *                2 s makes sun_run / sun_synchronize return SUN_ERR_TIMEOUT;
 *                16 = (SU(3) FP32) overrelaxation passes compute two links per
 *                thread with packed FP32 instructions ({add,sub,mul,fma}.f32x2),
 *                lane for lane the float operations: bitwise the same links.
 *  reunit_mode   where a sweep re-unitarizes (default 0); every link is
 *                re-unitarized once per re-unitarizing sweep in all three:
 *                0 = all links after the sweep's last step, as a pass of its own
 *                (the placement of Secs. 2-3); 1 = each link of the last step right
 *                after its update, inside the update kernel; 2 = spread over the
 *                steps: links in runs of 32 consecutive even/odd site indices
 *                (lex >> 1), run r re-unitarized right after its update in step
 *                r mod (n_heatbath + n_overrelax), inside the update kernel.
 *                Modes 1 and 2 are not built for FP64 with Nc >= 5 (SUN_ERR_UNSUPPORTED).
 *  wave_lag      with variant bit 8: t-slices the even units run ahead of the odd
 *                ones (0 = default 3; clamped to [1, Nt-1]); results do not
 *                depend on it.
 *  graph_sweeps  sweeps captured in one CUDA graph (sweeps per graph launch) by
 *                sun_run and by a batch built from this lattice first; 0 = 1,
 *                at most 64.  Results do not depend on it.  (With reunit_every
 *                > 1 sun_run launches one sweep at a time.)
 *  wave_skip_units  fault injection for tests of the bounded waits, 0 in normal
 *                use: every wavefront launch leaves out its first k units (even
 *                links of slice 0 first), so the odd units that need them wait
 *                until the 2 s limit and the lattice reports SUN_ERR_TIMEOUT;
 *                the links it updates are then not valid.
 */
typedef struct {
  int precision;
  int storage;
  int reunit_every;
  int block_threads;
  void* stream;
  void* device_buf;
  size_t device_buf_bytes;
  int use_graphs;
  int variant;
  int reunit_mode;
  int wave_lag;
  int wave_skip_units;
  int graph_sweeps;
} sun_options;

int sun_abi_version(void);
void sun_options_init(sun_options* opt);
const char* sun_status_string(sun_status s);
const char* sun_last_error(void); /* thread-local, "" when none */

/* Bytes of device memory a lattice needs (links, reduction scratch, observable
 * history, import/export staging).  0 if the arguments are invalid. */
size_t sun_footprint_bytes(int nc, const int dims[4], const sun_options* opt);

/* Create a lattice and initialise it (Sec. 3): cold start = every link the
 * identity; hot start = every link Haar-random in SU(Nc) (complex Gaussian matrix,
 * Gram-Schmidt, determinant phase), drawn with Philox counter (mu*V+lex, 0, k, 2).
 * beta = 2 Nc / g^2 (Eq. 3) must be >= 0.  The heatbath step counter starts at 0.
 * On success *out owns the lattice; on failure *out is NULL. */
sun_status sun_lattice_create(sun_lattice** out, int nc, const int dims[4], double beta,
                              int hot_start, uint64_t seed, const sun_options* opt);
void sun_lattice_destroy(sun_lattice* lat); /* syncs; NULL is a no-op */

/* One chessboard pass (Sec. 3): every link U_mu(x) with (x+y+z+t) % 2 == parity is
 * updated from its staple (Eq. 9) by the pseudo-heatbath (mode SUN_HEATBATH,
 * Eqs. 10-15, Kennedy-Pendleton/Creutz SU(2) subgroup draws, at most 64 attempts
 * per subgroup, using the current heatbath step counter) or by overrelaxation
 * (SUN_OVERRELAX, Eq. 17 per subgroup).  Does not advance the step counter. */
sun_status sun_update_pass(sun_lattice* lat, int mode, int mu, int parity);

/* The same pass with each updated link re-unitarized in FP64 (Sec. 2, as
 * sun_reunitarize) right after its update, inside the update kernel: the
 * placement reunit_mode 1 uses for the links of a sweep's last step.  Links
 * not updated by the pass are left as they are.  SUN_ERR_UNSUPPORTED where
 * reunit_mode 1 is not built (FP64 with Nc >= 5). */
sun_status sun_update_pass_reunit(sun_lattice* lat, int mode, int mu, int parity);

/* One sweep: n_heatbath heatbath steps then n_overrelax overrelaxation steps, a step
 * being the eight passes mu = 0..3 x (even, odd); then re-unitarization if this is a
 * reunit_every-th sweep.  Heatbath step s of the sweep uses counter value c + s,
 * and the counter advances by n_heatbath. */
sun_status sun_sweep(sun_lattice* lat, int n_heatbath, int n_overrelax);

/* n_sweeps sweeps as sun_sweep, each followed by the plaquette (if plaq_hist) and
 * the Polyakov loop (if poly_hist, re/im pairs) measured on the device; the
 * histories (n_sweeps and 2*n_sweeps doubles, host memory) are copied out at the
 * end.  With use_graphs, one sweep is captured as a CUDA graph and replayed.  Syncs. */
sun_status sun_run(sun_lattice* lat, int n_sweeps, int n_heatbath, int n_overrelax,
                   double* plaq_hist, double* poly_hist);

/* Re-unitarize every link in FP64 (Sec. 2): Nc=2 normalise the first row and
 * rebuild the second; Nc=3 Gram-Schmidt rows 0,1 and row 2 = conj(row0 x row1);
 * Nc>3 Gram-Schmidt all rows, then the last row times conj(det). */
sun_status sun_reunitarize(sun_lattice* lat);

/* <P> = sum_x sum_{mu<nu} ReTr P_{mu nu}(x) / (6 V Nc) (Eq. 4), products in the
 * storage precision, accumulated in FP64 with a fixed reduction order.  Syncs. */
sun_status sun_plaquette(sun_lattice* lat, double* out);

/* Polyakov loop L = sum_{x,y,z} Tr prod_{t=0}^{Nt-1} U_3(x,y,z,t) / (Nc Nx Ny Nz),
 * accumulated in FP64 (not defined in the paper; the usual order-parameter
 * definition).  Syncs. */
sun_status sun_polyakov_loop(sun_lattice* lat, double* re, double* im);

/* Copy all links to / from host memory in canonical order (n_doubles must equal
 * 8*Nc*Nc*V; the buffer 16-byte aligned).  Export rebuilds the third row of
 * 12-real storage; import of a 12-real lattice keeps rows 0 and 1 only.
 * Page-locked host memory is read or written directly by the conversion kernel
 * (mapped into the device address space).  Pageable memory is read directly too
 * where the device reaches it through the host's page tables (a Grace host on
 * NVLink-C2C); otherwise, and for every export to pageable memory, it goes
 * through a device staging buffer in chunks.  Both sync. */
sun_status sun_export_links(sun_lattice* lat, double* host, size_t n_doubles);
sun_status sun_import_links(sun_lattice* lat, const double* host, size_t n_doubles);

/* Health of the links (no counterpart in the paper; a diagnostic): over all 4V
 * stored links, in FP64 of the stored values (two-row storage: with the
 * rebuilt third row), the largest entry |(U U^+ - 1)_ij|, the largest
 * |det U - 1|, and the number of links with a NaN or infinite entry (those are
 * left out of the two maxima).  Syncs. */
sun_status sun_check_links(sun_lattice* lat, double* max_unitarity_dev, double* max_det_dev,
                           uint64_t* nonfinite);

/* The compact host format: for every link in canonical order the rows
 * 0 .. storage/(2 Nc) - 1 that the storage format keeps, as (re, im) pairs in
 * the lattice's precision (the payload of configuration files): 4V x stored link
 * bytes (sun_lattice_info.links_bytes).  Exact both ways: the stored values
 * themselves.  SU(2) quaternion storage: row 0 = (a0 + i a3, a2 + i a1).  The
 * buffer must be 16-byte aligned; page-locked host memory is read or written
 * directly by the conversion kernel, and pageable memory as for
 * sun_import_links / sun_export_links (read in place where the device can,
 * written through the staging buffer).  Both sync. */
sun_status sun_export_stored(sun_lattice* lat, void* host, size_t bytes);
sun_status sun_import_stored(sun_lattice* lat, const void* host, size_t bytes);

/* Random state: the heatbath step counter (the seed is fixed at creation). */
sun_status sun_get_heatbath_step(sun_lattice* lat, uint64_t* step); /* syncs */
sun_status sun_set_heatbath_step(sun_lattice* lat, uint64_t step);
sun_status sun_set_beta(sun_lattice* lat, double beta);
sun_status sun_synchronize(sun_lattice* lat);

typedef struct {
  int nc, precision, storage, reserved;
  int dims[4];
  double beta;
  uint64_t seed;
  size_t link_bytes;     /* bytes of one stored link                     */
  size_t links_bytes;    /* bytes of all 4V links                        */
  size_t footprint;      /* device bytes held by the lattice             */
  void* links;           /* device address of the link storage           */
  void* stream;          /* cudaStream_t the lattice enqueues on         */
} sun_lattice_info;
sun_status sun_get_info(const sun_lattice* lat, sun_lattice_info* info);

/* ---------------------------------------------------------------------------
 * Configuration files.  The paper stores the generated configurations (Sec. 3);
 * this format also carries the chain's state, so that a saved lattice resumes
 * bitwise: links, beta, seed, heatbath step counter and sweep count.
 *
 * Layout (little-endian): a 128-byte header, then the payload.
 *   header: char magic[8] = "SUNCFG01", then sun_config_header as laid out below
 *   payload: every link in canonical order (mu, t, z, y, x), for each the rows
 *   0 .. rows-1 of the matrix as (re, im) pairs, in the lattice's precision
 *   (float or double); rows = storage / (2 Nc): the rows the storage format
 *   keeps (SU(2) quaternion storage: row 0 = (a0 + i a3, a2 + i a1); SU(3)
 *   two-row: rows 0, 1; full storage: all rows).  FP32 links are stored exactly.
 *   checksum: FNV-1a (64-bit offset basis and prime) over the payload read as
 *   little-endian 64-bit words (the payload is a multiple of 8 bytes).
 */
typedef struct {
  uint32_t version;        /* 1 */
  int32_t nc, precision, storage;
  int32_t dims[4];
  double beta;
  uint64_t seed;
  uint64_t heatbath_step;
  uint64_t sweeps_done;    /* sets the re-unitarization cadence (reunit_every) */
  uint64_t payload_bytes;  /* 4V * rows * Nc * 2 * (precision / 8) */
  uint64_t checksum;
  uint8_t reserved[40];
} sun_config_header;       /* 120 bytes, stored right after the 8-byte magic */

/* Write the lattice and its chain state to path (created or truncated).
 * Streams through the lattice's staging buffer.  Syncs. */
sun_status sun_save_config(sun_lattice* lat, const char* path);

/* Read a file written by sun_save_config into a lattice of the same nc, dims,
 * precision and storage (SUN_ERR_ARG otherwise): links, beta, seed, heatbath
 * step and sweep count.  The whole payload is read and checksummed before the
 * lattice is touched; a mismatch returns SUN_ERR_ARG with the lattice
 * unchanged.  Syncs. */
sun_status sun_load_config(sun_lattice* lat, const char* path);

/* Read and check a file's header; with verify != 0 also read the payload and
 * check its size and checksum.  Host only: needs no GPU. */
sun_status sun_read_config_header(const char* path, int verify, sun_config_header* out);

/* ---------------------------------------------------------------------------
 * Batches: many independent chains swept together.
 * A batch references existing lattices (they must outlive it) of possibly
 * different Nc, extents, beta and seed.  Lattices with the same (Nc, storage,
 * precision) form a group; each chessboard pass, re-unitarization and
 * observable of a group is one kernel launch over all its chains (block ->
 * chain table), and groups run on their own streams so that their kernels
 * overlap.  Each chain evolves exactly as it would alone: same kernels per link,
 * its own seed and heatbath step counter, and per-chain FP64 observable sums
 * in a fixed order.  All lattices must share reunit_every (0 or 1) and
 * reunit_mode; a batch uses the kernel variant and block size of each group's
 * first lattice.
 */
typedef struct sun_batch sun_batch;

/* stream: cudaStream_t the batch synchronises with (NULL = one the batch creates);
 * use_graphs: sun_batch_run captures one batch sweep as a CUDA graph and replays it. */
sun_status sun_batch_create(sun_batch** out, sun_lattice* const* lattices, int n, void* stream,
                            int use_graphs);

/* n_sweeps sweeps of every chain as sun_run (n_heatbath heatbath + n_overrelax
 * overrelaxation steps, re-unitarization per the lattices' options), each followed
 * by the plaquette (plaq: n_sweeps x n doubles, row = sweep, column = the chain's
 * position in the create call) and the Polyakov loop (poly: n_sweeps x n x 2)
 * when the pointers are not NULL.  Each chain's heatbath counter advances by
 * n_sweeps * n_heatbath.  Waits for the lattices' own streams first.  Syncs. */
sun_status sun_batch_run(sun_batch* b, int n_sweeps, int n_heatbath, int n_overrelax, double* plaq,
                         double* poly);
void sun_batch_destroy(sun_batch* b); /* syncs; the lattices are not touched */

/* ---------------------------------------------------------------------------
 * t-slab decomposition (Sec. 3: the paper splits the lattice in the time
 * direction over GPUs and exchanges the border slices).  The lattice is cut
 * into n_slabs slabs of Nt / n_slabs consecutive t-slices (an even number);
 * each slab is a lattice of its own with one halo slice on each side.  After
 * every chessboard pass (direction mu, parity) each slab copies the two
 * boundary slices of that (mu, parity) block into its neighbours' halos, so the
 * next pass reads exactly the links the whole lattice would hold.  Random
 * numbers are keyed by each link's index in the whole lattice, so the slabs
 * produce bitwise the links of one lattice with the same seed; the plaquette
 * and Polyakov loop agree to FP64 summation order.  All slabs live on the
 * current device and share one stream (a stand-in for one GPU per slab: the
 * halo copies are device-to-device transfers of contiguous slices).  Options
 * as for a lattice, except device_buf (must be NULL) and reunit_every (0 or 1).
 */
typedef struct sun_slabs sun_slabs;
sun_status sun_slabs_create(sun_slabs** out, int nc, const int dims[4], int n_slabs, double beta,
                            int hot_start, uint64_t seed, const sun_options* opt);
void sun_slabs_destroy(sun_slabs* slabs); /* syncs; NULL is a no-op */
/* n_sweeps sweeps as sun_run, with the histories of the whole lattice.  Syncs. */
sun_status sun_slabs_run(sun_slabs* slabs, int n_sweeps, int n_heatbath, int n_overrelax,
                         double* plaq_hist, double* poly_hist);
/* the whole lattice in canonical order, as sun_export_links / sun_import_links (pageable host memory). */
sun_status sun_slabs_export_links(sun_slabs* slabs, double* host, size_t n_doubles);
sun_status sun_slabs_import_links(sun_slabs* slabs, const double* host, size_t n_doubles);

/* ---------------------------------------------------------------------------
 * Autotuning.  The paper tunes its kernels by hand for its GPU (Sec. 3: threads
 * per block, storage format, read path); here the configuration is measured on
 * the GPU at hand.  Scratch lattices of the requested shape (hot start) are
 * swept with each candidate configuration through sun_run / sun_batch_run and
 * the fastest is kept.  The search goes one option at a time, each stage
 * starting from the best of the previous one:
 *   1. kernel shape: block_threads 64, 128, 256; variant bit 1 (SU(3) FP32, and
 *      SU(4) FP32 for a single lattice);
 *      per-link or row-parallel kernel (bit 4, Nc 4 and 6); with
 *      SUN_TUNE_TWO_ROW also bit 2
 *   2. with SUN_TUNE_STORAGE: storage (Nc = 2: 4 or 8 reals, Nc = 3: 12 or 18)
 *   3. with SUN_TUNE_REUNIT_MODE: reunit_mode 0, 1, 2
 *   4. variant bit 8 (wavefront launches), for kernels that have that form
 *   5. graph_sweeps 1, 4, 16 (sweeps per graph launch), with use_graphs
 * Bits 1, 4, 8 and 16, block_threads, wave_lag and graph_sweeps leave the results bitwise
 * unchanged; storage, reunit_mode and bit 2 change them at the level of FP32
 * rounding (results stay within the FP32 tolerance of the FP64 oracle).
 */
enum {
  SUN_TUNE_STORAGE = 1,
  SUN_TUNE_REUNIT_MODE = 2,
  SUN_TUNE_TWO_ROW = 4
};

/* Tune for one lattice of shape (nc, dims) at coupling beta swept with
 * n_heatbath + n_overrelax steps per sweep.  *opt supplies precision,
 * reunit_every, use_graphs, stream, wave_lag, and storage / reunit_mode where
 * those are not tuned; on success the fastest configuration is written back
 * into *opt (block_threads, variant, graph_sweeps and the tuned fields) and, if
 * ms_per_sweep is not NULL, its time per sweep.  device_buf must be NULL.
 * Results are cached for the process by (GPU name and multiprocessor count,
 * shape, beta, steps, flags, fixed options): a repeated call returns at once.
 * If the environment variable SUN_TUNE_CACHE names a file, results are also
 * read from it (first call) and appended to it, one line per result.  Scratch lattices are
 * created one at a time (sun_footprint_bytes each).  Syncs; takes about 30 ms
 * of sweeps per candidate, 6 to 12 candidates. */
sun_status sun_autotune(int nc, const int dims[4], double beta, int n_heatbath, int n_overrelax, int flags,
                        sun_options* opt, double* ms_per_sweep);

/* The same for a batch of n chains (nc[i], dims[4i .. 4i+3], beta[i]) swept
 * together by sun_batch_run; every chain of the batch is to be created with the
 * returned options.  The storage format is tuned only when all chains share Nc.
 * The scratch lattices of all n chains exist at the same time. */
sun_status sun_autotune_batch(int n, const int* nc, const int* dims, const double* beta, int n_heatbath,
                              int n_overrelax, int flags, sun_options* opt, double* ms_per_sweep);

/* Plaquette of link storage the caller already holds, with no allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they measure -- code confined to a memory
 * arena it does not own (a framework that hands out fixed buffers and forbids
 * cudaMalloc after start-up), latency-critical loops that cannot afford an
 * allocation's implicit synchronisation.
 *  links      device address of link storage in this library's layout (e.g.
 *             sun_lattice_info.links of a lattice with the same nc, dims,
 *             precision, storage); read only
 *  nc, dims, precision, storage  as for sun_lattice_create (storage 0 = default)
 *  out        device address of one double that receives <P>, normalised as
 *             sun_plaquette; the caller owns it
 *  stream     cudaStream_t to enqueue on (NULL = the legacy default stream); the
 *             call is asynchronous and does not synchronise
 * Calls no cudaMalloc, cudaFree or allocating library routine.  The reduction
 * scratch is a fixed array in the library's device image: 512 KiB + 256 B on every
 * GPU that loads the library, held until the process exits, so at most
 * 16,777,216 sites (65,536 blocks of 256 sites) -- larger lattices are rejected
 * with SUN_ERR_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current): make that first call
 * before any stream capture.  Every call shares the array and re-arms its
 * counter: calls that overlap on the GPU (other streams, other host threads
 * without ordering) race -- order them on one stream. */
sun_status sun_plaquette_noalloc(const void* links, int nc, const int dims[4], int precision,
                                 int storage, double* out, void* stream);

/* Self-test of the FP32 <-> FP64 conversions the kernels use (no counterpart in
 * the paper; a diagnostic).  The re-unitarization kernels (sun_reunitarize)
 * convert links between the FP32 storage and FP64 with integer operations on
 * the IEEE 754 encodings, because GB300 runs its conversion instructions at its
 * FP64 rate.  This compares them bit for bit with the
 * hardware conversions on the current device: all 2^32 float encodings through
 * float -> double, and n double encodings drawn from seed (exponents across and
 * around the float's normal range, and rounding ties) through double -> float.
 *  result[0]  float -> double mismatches     result[1]  double -> float mismatches
 *  result[2]  smallest mismatching float encoding, result[3] smallest mismatching
 *             double encoding (UINT64_MAX when there is none)
 * Allocates 32 bytes of device memory for the call; uses the legacy default
 * stream; syncs.  SUN_ERR_ARG if result is NULL, SUN_ERR_CUDA on a CUDA error. */
sun_status sun_selftest_conversions(uint64_t n, uint64_t seed, uint64_t result[4]);

#ifdef __cplusplus
}
#endif
#endif /* SUN_H */
