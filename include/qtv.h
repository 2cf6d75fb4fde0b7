/*
 * qtv.h -- C ABI of libqtv: GPU vortex-core identification and sub-grid
 * localization on a 3-D grid of a complex wave function psi.
 *
 * The two stages follow "Vectorizing Quantum Turbulence Vortex-Core Lines for
 * Real-Time Visualization" (Liu, Xiong, Liu; arXiv 1911.12070):
 *
 *   identification -- circulation-based vortex identification, Sec. 2.2.2,
 *     Eq. 5: C = closed-path integral of grad(sigma) . dl, |C| = 2 pi where the
 *     path encloses a vortex core and 0 elsewhere.  Here the path is every
 *     plaquette (unit square) of the three axis-aligned orientations, and the
 *     result is the integer winding W = C / (2 pi) of each plaquette.
 *   localization -- density-guided local optimisation, Sec. 3.3.3, Eq. 6:
 *     x* = argmin rho(x), rho = |Phi|^2 (Eq. 3), with Phi linearly
 *     interpolated between grid nodes (Sec. 5).  Here the search domain of
 *     each sample is its pierced plaquette, where the bilinear interpolant has
 *     exactly one zero when W = +-1.
 *   direction -- each sample carries W, whose sign gives the direction of the
 *     line by the right-hand rule about the plaquette normal (Sec. 3.4).
 *
 * Conventions shared by every entry point
 *   psi      device pointer, complex64 interleaved (re, im) as two float32,
 *            nx*ny*nz elements, x fastest: node (i,j,k) is element
 *            (k*ny + j)*nx + i.  At least 8-byte aligned (16-byte alignment
 *            and even nx enable 16-byte vector loads).
 *   faces    named by the minimum corner (i,j,k) and orientation o:
 *            o = 0: xy plaquette, normal +z, loop (i,j)->(i+1,j)->(i+1,j+1)->(i,j+1)
 *            o = 1: yz plaquette, normal +x, loop (j,k)->(j+1,k)->(j+1,k+1)->(j,k+1)
 *            o = 2: zx plaquette, normal +y, loop (k,i)->(k+1,i)->(k+1,i+1)->(k,i+1)
 *            A face exists iff its four corners are in the grid (no periodic
 *            wrap).  face id = (((k*ny + j)*nx + i) << 2) | o, a uint64.
 *   streams  every call is asynchronous on the given cudaStream_t (passed as
 *            void*; NULL = legacy default stream) unless stated otherwise.
 *   memory   the caller owns every input and output buffer.  The handle owns
 *            only its workspace (staging for stream compaction, segment tables).
 *   errors   every call returns a status code; nothing throws across the ABI.
 *            qtv_last_error_string() describes the last failure of the calling
 *            thread.  Invalid arguments are rejected on the host before any
 *            launch; device-side conditions are reported through device memory.
 */
#ifndef QTV_H
#define QTV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QTV_API __attribute__((visibility("default")))
#else
#define QTV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define QTV_OK 0
#define QTV_WARN_NONFINITE 1  /* not returned by asynchronous calls; see qtv_stats */
#define QTV_ERR_ARG (-1)      /* invalid argument (null pointer, bad size, misalignment) */
#define QTV_ERR_CAPACITY (-2) /* workspace or output too small; required size reported */
#define QTV_ERR_CUDA (-3)     /* a CUDA runtime call failed */
#define QTV_ERR_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define QTV_ERR_STATE (-5)    /* call not valid in the handle's current state */

/* value of *count after a call whose bounded device-side wait gave up
 * (the outputs are then unusable; the binding raises QTV_ERR_TIMEOUT) */
#define QTV_COUNT_TIMEOUT 0xFFFFFFFFFFFFFFFFull

/* localization modes */
#define QTV_PLAIN 0   /* closed-form zero of the bilinear interpolant + Newton polish */
#define QTV_LEARNED 1 /* learned locator with plain fallback (needs loaded weights) */

/* per-sample flag bits */
#define QTV_FLAG_ANOMALOUS 1u /* |W| != 1, or no zero of the interpolant inside the face */
#define QTV_FLAG_FALLBACK 2u  /* learned prediction rejected; plain result used */
#define QTV_FLAG_LEARNED 4u   /* position predicted by the learned locator */

typedef struct qtv_handle_s* qtv_handle;

/* Grid geometry.  h and origin only scale and shift output positions:
 * node (i,j,k) sits at origin + h*(i,j,k).  periodic must be 0.  Sizes: nx up
 * to 2048, any ny and nz (node indices are 64-bit, so grids beyond 2^32
 * nodes such as 2048^3 work).  Even nx with a 16-byte aligned field takes the
 * staged sweeps (the bit-sliced default up to 2048 columns, the nibble sweep
 * up to 1024); odd nx or an 8-byte aligned field takes the register sweep. */
typedef struct {
  int32_t nx, ny, nz;
  float h;
  float origin[3];
  uint32_t periodic;
} qtv_grid;

/* Optional statistics of one identification call (device memory, written by
 * the call).  faces_scanned = existing faces; pierced = faces with W != 0;
 * ambiguous = faces with an edge phase difference within about 1e-4 rad of
 * +-pi (FP32 test); zero_node_faces = faces with a corner where psi == 0;
 * nonfinite_faces = faces with a NaN/Inf corner (their W is forced to 0). */
typedef struct {
  uint64_t faces_scanned;
  uint64_t pierced;
  uint64_t ambiguous;
  uint64_t zero_node_faces;
  uint64_t nonfinite_faces;
  uint64_t anomalous;
  uint64_t fallbacks;
  uint64_t reserved;
} qtv_stats;

/* One emitted core sample (32 bytes, host memory). */
typedef struct {
  float x, y, z;   /* position, origin + h * grid coordinates */
  float resid;     /* |psi_interp|^2 at the position (Eq. 6 objective) */
  uint64_t face_id;
  int8_t winding;  /* W of the pierced plaquette: direction by the right-hand rule */
  uint8_t flags;   /* QTV_FLAG_* */
  uint16_t reserved0;
  uint32_t reserved1;
} qtv_sample;

/* Library version, (major << 16) | minor. */
QTV_API int qtv_version(void);

/* Text of the last error on the calling thread ("" if none).  The pointer
 * stays valid until the thread's next failing call. */
QTV_API const char* qtv_last_error_string(void);

/* Create a handle bound to CUDA device `device` (made current for the call).
 * Allocates no large workspace; see qtv_reserve.  *out receives the handle. */
QTV_API int qtv_create(qtv_handle* out, int device);

/* Free the handle and its workspace.  Synchronises the handle's device.
 * NULL is accepted (no-op). */
QTV_API int qtv_destroy(qtv_handle h);

/* Size the handle's workspace for grids up to `grid` and up to max_faces
 * pierced faces per identification call.  Synchronous (cudaMalloc).  Calls
 * made later with larger sizes grow the workspace the same way, so call this
 * first when later calls are captured into a CUDA graph. */
QTV_API int qtv_reserve(qtv_handle h, const qtv_grid* grid, uint64_t max_faces);

/*
 * Identification (Sec. 2.2.2, Eq. 5) of every plaquette of the grid.
 *
 *   psi       device, complex64 field as above (read only).
 *   face_ids  device, uint64[capacity]: ids of the faces with W != 0, in
 *             ascending face-id order.
 *   winding   device, int8[capacity]: W of each listed face.
 *   capacity  length of face_ids / winding.
 *   count     device, one uint64: receives the number of faces with W != 0.
 *             If *count > capacity the face outputs are incomplete and must
 *             not be used: retry with capacity >= *count (the Python binding
 *             does this).  capacity = 0 with NULL outputs counts only.
 *   stats     device qtv_stats or NULL.  NULL selects the fastest kernel.
 *
 * W is the sum over the four directed loop edges of the integer branch
 * crossing of arg(psi), so that 2 pi W equals the sum of the wrapped phase
 * differences arg(psi_b * conj(psi_a)) in (-pi, pi] (the discrete Eq. 5) up to
 * rounding of those differences; it equals the FP64 definition on every face
 * whose edge differences lie at least 1e-4 rad from +-pi.  A node with psi == 0
 * exactly is given phase 0.  A face with a NaN/Inf corner gets W = 0.
 * Returns QTV_ERR_ARG for bad arguments; device results are asynchronous.
 */
QTV_API int qtv_identify(qtv_handle h, const qtv_grid* grid, const void* psi, uint64_t* face_ids,
                 int8_t* winding, uint64_t capacity, uint64_t* count, qtv_stats* stats,
                 void* stream);

/*
 * Localization (Sec. 3.3.3, Eq. 6) of a list of pierced faces.
 *
 *   face_ids, winding  device, n entries (as produced by qtv_identify).
 *   n        host upper bound on the number of faces (buffer length).
 *   n_dev    optional device uint64: if not NULL the call processes
 *            min(n, *n_dev) faces, so it can follow qtv_identify without a
 *            host synchronisation.
 *   mode     QTV_PLAIN or QTV_LEARNED.
 *   fallback_resid  learned mode only: predictions whose interpolated |psi|^2,
 *            divided by the neighbourhood mean |psi|^2, exceeds this are
 *            replaced by the plain result (QTV_FLAG_FALLBACK).
 *   xyz      device float[3*n]: sample positions, origin + h*(grid coords).
 *   resid    device float[n]: |psi_bilinear|^2 at the sample.
 *   flags    device uint8[n]: QTV_FLAG_* bits.
 */
QTV_API int qtv_localize(qtv_handle h, const qtv_grid* grid, const void* psi, const uint64_t* face_ids,
                 const int8_t* winding, uint64_t n, const uint64_t* n_dev, int mode,
                 float fallback_resid, float* xyz, float* resid, uint8_t* flags, void* stream);

/*
 * Identification and plain localization in one call: the result of
 * qtv_identify followed by qtv_localize(QTV_PLAIN, n_dev = count) on its
 * faces, enqueued together without a host synchronisation.  Outputs as in
 * those calls, each with `capacity` entries; *count as in qtv_identify.
 */
QTV_API int qtv_identify_localize(qtv_handle h, const qtv_grid* grid, const void* psi,
                                  uint64_t* face_ids, int8_t* winding, uint64_t capacity,
                                  uint64_t* count, float* xyz, float* resid, uint8_t* flags,
                                  qtv_stats* stats, void* stream);

/*
 * Emission (Sec. 3.4, direction by the right-hand rule): pack n samples into
 * caller-owned host memory `host_out` (qtv_sample[n]; pinned memory makes the
 * copy asynchronous).  Samples keep the order of the inputs (ascending face
 * id when they come from qtv_identify).  The copy is complete when `stream`
 * reaches this point; synchronise before reading host_out.
 */
QTV_API int qtv_emit_samples(qtv_handle h, uint64_t n, const uint64_t* face_ids, const int8_t* winding,
                     const float* xyz, const float* resid, const uint8_t* flags,
                     qtv_sample* host_out, void* stream);

/*
 * Identification and plain localization from host memory, end to end: the
 * field is copied from the caller's host buffer into one of two device copies
 * the handle keeps, identified and localized as by qtv_identify_localize, and
 * the samples (qtv_sample records, ascending face id) and their count are
 * copied back to the caller's host buffers.
 *
 *   psi_host    host complex64 field (conventions above); page-locked memory
 *               (cudaHostAlloc / cudaHostRegister) makes the copy asynchronous.
 *   capacity    samples kept per call; host_out receives `capacity` records, of
 *               which the first *host_count are the samples (if *host_count
 *               exceeds capacity the list is incomplete: call again with a
 *               larger capacity).
 *   host_out    host qtv_sample[capacity]; host_count: host uint64.
 * Asynchronous on `stream`: results are complete when the stream reaches the
 * end of the call.  Consecutive calls alternate between the two device copies
 * and copy the field on a stream of the handle, so the copy of one call
 * overlaps the identification of the previous one; the caller gives
 * consecutive calls different host_out / host_count buffers (or synchronises
 * in between).  The device copies (2 x the field) and output buffers are
 * handle workspace, allocated on first use (a synchronising step).
 */
QTV_API int qtv_identify_localize_host(qtv_handle h, const qtv_grid* grid, const void* psi_host,
                                       uint64_t capacity, qtv_sample* host_out,
                                       uint64_t* host_count, void* stream);

/*
 * Identification without any allocation (the paper has no counterpart; this
 * is a deployment variant of qtv_identify).
 *
 * Some callers cannot allocate device memory at call time: engines that
 * reserve the whole GPU up front through their own allocator, plug-ins that
 * must not touch the device heap, and latency-critical loops where cudaMalloc
 * or cudaFree would synchronise the device.  For them this entry point takes
 * no handle and allocates nothing: its scratch lives in one fixed file-scope
 * device array of the library (about 64 MiB, held on every GPU that loads
 * libqtv until the process exits).  The caller still passes psi and the
 * outputs, with the same meaning as in qtv_identify (no statistics).
 *
 * Limits: capacity <= QTV_STATIC_MAX_FACES, nz * ceil(ny / 7) <=
 * QTV_STATIC_MAX_SEGMENTS and nz * ceil(ny / 7) * ceil(nx / 64) <=
 * QTV_STATIC_MAX_WARP_SEGMENTS (enough for 512^3 tangles); larger requests
 * are rejected with QTV_ERR_ARG and a message naming the limit.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before capturing any stream.  The call uses the current device.  The
 * address is kept for the life of the process: calls after cudaDeviceReset
 * on that device are not supported.  Odd nx, or psi aligned to 8 but not 16
 * bytes, runs the register sweep instead of the staged one, within the same
 * limits.
 * Every call shares the one array, and the array keeps the last call's
 * contents (each call clears what must start at zero): calls that may
 * overlap on the GPU (different streams, or different host threads on the
 * same device) race and must be serialised by the caller.
 */
#define QTV_STATIC_MAX_FACES (1u << 21)
#define QTV_STATIC_MAX_SEGMENTS (1u << 17)
#define QTV_STATIC_MAX_WARP_SEGMENTS (1u << 19)
QTV_API int qtv_identify_static(const qtv_grid* grid, const void* psi, uint64_t* face_ids,
                                int8_t* winding, uint64_t capacity, uint64_t* count,
                                void* stream);

/*
 * Learned locator (the paper has no counterpart: it is trained on positions
 * made by the plain localization, Sec. 3.3.3 / Eq. 6, which stays its fallback
 * and the judge of its error).  A 128-256-256-3 MLP (ReLU) maps the encoded
 * 4x4x4 neighbourhood of a pierced face to its face coordinates (u, v, n);
 * dense layers use BF16 tensor cores with FP32 accumulation.
 *
 * Encoding (qtv_locator_encode): block node (a, b, c) in 0..3 is grid node
 * min_corner + (a-1) e_u + (b-1) e_v + (c-1) e_n in the face frame
 * (u, v, n) = (x, y, z), (y, z, x), (z, x, y) for xy, yz, zx faces; psi is
 * conjugated for W = -1, multiplied by conj(P0)/|P0| with P0 the value at
 * the face's minimum corner (block node (1, 1, 1)), and divided by the RMS of
 * |psi| over the block.
 * x is BF16 [n][128] with index ((c*4 + b)*4 + a)*2 + {0: Re, 1: Im};
 * ok[f] = 0 for faces whose block leaves the grid; rms[f] = the RMS.
 *
 * Parameters: QTV_LOCATOR_PARAMS FP32 values: W1 [256][128], b1 [256],
 * W2 [256][256], b2 [256], W3 [3][256], b3 [3] (weights as [out][in]).
 * Adam state: first then second moments, 2 * QTV_LOCATOR_PARAMS values.
 * Training: loss = mean over the batch of |y - target|^2; one Adam step
 * (beta 0.9 / 0.999, eps 1e-8) per qtv_locator_train_step; batch sizes are
 * positive multiples of 64.  x, targets, y, grads and loss are device memory.
 * Inference is qtv_localize(mode = QTV_LEARNED): predictions outside the face
 * or with |psi_bilinear(u, v)|^2 / rms^2 > fallback_resid are replaced by the
 * plain result (QTV_FLAG_FALLBACK); accepted ones carry QTV_FLAG_LEARNED.
 * Checkpoints (qtv_locator_save / _load) hold the step count, parameters and
 * Adam moments with an FNV-1a checksum; loading resumes training exactly.
 */
#define QTV_LOCATOR_PARAMS 99587
QTV_API int qtv_locator_init(qtv_handle h, uint64_t seed);
QTV_API int qtv_locator_get(qtv_handle h, float* params, float* adam, uint64_t* step);
QTV_API int qtv_locator_set(qtv_handle h, const float* params, const float* adam, uint64_t step);
QTV_API int qtv_locator_encode(qtv_handle h, const qtv_grid* grid, const void* psi,
                               const uint64_t* face_ids, const int8_t* winding, uint64_t n,
                               const uint64_t* n_dev, uint16_t* x, uint8_t* ok, float* rms,
                               void* stream);
QTV_API int qtv_locator_forward(qtv_handle h, const uint16_t* x, uint64_t n, float* y,
                                void* stream);
QTV_API int qtv_locator_gradients(qtv_handle h, const uint16_t* x, const float* targets,
                                  uint64_t n, float* grads, float* loss, void* stream);
QTV_API int qtv_locator_train_step(qtv_handle h, const uint16_t* x, const float* targets,
                                   uint64_t n, float lr, float* loss, void* stream);
QTV_API int qtv_locator_save(qtv_handle h, const char* path);
/* Tensor-core path of the network: 0 = mma.sync layer kernels, 1 = tcgen05
 * (the default): inference (qtv_locator_forward and learned localization) in
 * one kernel for the whole network (accumulators and the hidden activations
 * in tensor memory), training (qtv_locator_gradients, qtv_locator_train_step)
 * with every dense contraction - forward, data gradient and weight gradients
 * - as tcgen05 GEMMs with accumulators in tensor memory (weight gradients
 * split along the batch and summed in a fixed order).  Both paths use BF16
 * operands with FP32 accumulation; results agree to accumulation order.
 * On path 1, qtv_locator_forward reads x by tensor copies: x must be 16-byte
 * aligned and n below 2^31 (else QTV_ERR_ARG). */
QTV_API int qtv_locator_set_tensor_path(qtv_handle h, int path);
QTV_API int qtv_locator_load(qtv_handle h, const char* path);

/*
 * Shape of the identification sweep used by this handle's single-snapshot
 * calls.  variant 0: nibble sweep (7-row bands, 64 columns per warp, warps
 * per tile 1..16, 0 = one tile per row); variant 1: bit-sliced sweep (16-row
 * bands, 31 columns per warp, warps per tile 2, 4 or 8, 0 = 4; stages 2 or 3
 * shared-memory ring slots, 0 = 3; rows wider than 32 warps of tiles fall back
 * to variant 0); -1: the library default.  ctas_per_sm caps resident CTAs per
 * SM (0 = as many as fit).  Both variants give identical results.
 */
QTV_API int qtv_configure_sweep(qtv_handle h, int variant, int warps_per_tile, int stages,
                                int ctas_per_sm);

/*
 * Failure injection for tests of the bounded device waits (no paper
 * counterpart).  Every later identification of this handle runs its segment
 * scan with look-back tile `hold_tile` never publishing its state (-1 = none),
 * and with look-back waits that give up after `spin_cycles` SM cycles (0 = the
 * default, about 2^32).  A wait that gives up ends its kernel normally, sets
 * the reported face count to QTV_COUNT_TIMEOUT and leaves the CUDA context
 * usable; the face list of that call is then meaningless (faces are still
 * written only below capacity).  qtv_inject_scan_hold(h, -1, 0) restores
 * normal operation.  Returns QTV_ERR_ARG for a NULL handle, hold_tile < -1 or
 * a negative spin limit.
 */
QTV_API int qtv_inject_scan_hold(qtv_handle h, int64_t hold_tile, int64_t spin_cycles);

/*
 * Batches of snapshots.  Identification (Sec. 2.2.2, Eq. 5) and localization
 * (Sec. 3.3.3, Eq. 6) of up to QTV_BATCH_MAX snapshots of different grid
 * sizes in one pass: persistent sweep launches whose CTAs take contiguous
 * ranges of the (plane, band, x tile) units of many snapshots (one launch for
 * all snapshots at a common tile width, or one per group of snapshots of equal
 * row width, serial or concurrent), then one scan, one expand and one
 * localization launch over the concatenated face list.
 * The sequence is captured into a CUDA graph on the first qtv_batch_run and
 * replayed by later calls with the same outputs and mode.
 *
 * qtv_batch_plan: grids[i] / psis[i] (device, complex64, x fastest, 16-byte
 * aligned, even nx <= 2048, periodic = 0; rows wider than 1024 columns only
 * with the bit-sliced sweep) must stay valid and unchanged in
 * place until the next plan or qtv_destroy (new data may be written into the
 * same buffers between runs).  The call runs a counting pass, then picks the
 * sweep shape (warps per x tile, resident CTAs per SM, z-block height) by
 * timing candidates on these fields, unless tune_cache names a text file that
 * holds a shape for this device and these grid sizes; a newly timed shape is
 * appended to that file (tune_cache may be NULL).  Each line of the file is
 * "qtv-tune-v3 <key> <variant> <warps per tile, 0 = per snapshot> <CTAs per
 * SM, 0 = max> <z-block factor> <concurrent 0/1> <stages> <ms>" (variant and
 * stages as for qtv_configure_sweep); the last line whose key matches wins,
 * and the key "*" matches every batch (a pinned shape).
 * Synchronizes `stream`.
 *
 * qtv_batch_run: face_ids / winding [capacity] receive the faces of all
 * snapshots, snapshot i in [offsets[i], offsets[i+1]) in ascending face-id
 * order (face ids are snapshot-local); offsets (device, n + 1 entries)
 * receives the slice starts and the total in offsets[n]
 * (QTV_COUNT_TIMEOUT when a bounded wait gave up).  A total above capacity
 * means outputs were truncated: grow and run again.  xyz [capacity][3],
 * resid and flags (all NULL to skip localization) receive the positions
 * (mode QTV_PLAIN or QTV_LEARNED, as qtv_localize).  Asynchronous on stream.
 */
#define QTV_BATCH_MAX 32
typedef struct {
  uint64_t nodes;         /* grid nodes of all snapshots */
  uint64_t faces;         /* pierced faces found by the counting pass */
  int32_t warps_per_tile; /* chosen shape: tiles of 64 * warps_per_tile columns for every
                             snapshot, or 0: each snapshot one tile as wide as its row */
  int32_t tile_columns;   /* owned columns per tile: 64 * warps_per_tile (variant 0; 0 when
                             per snapshot) or 31 * warps_per_tile (variant 1) */
  int32_t ctas_per_sm;    /* cap on resident CTAs per SM (0: as many as fit) */
  float zscale;           /* factor on the z-block height */
  int32_t concurrent;     /* 1: sweeps of the width groups run concurrently */
  int32_t variant;        /* sweep variant (qtv_configure_sweep) */
  int32_t stages;         /* ring stages of the bit-sliced sweep */
  int32_t sweeps;         /* sweep launches (width groups) */
  int32_t grid;           /* CTAs of all sweep launches */
  int32_t source;         /* 1: tune cache, 2: timed now */
  int32_t candidates;     /* shapes timed (source 2) */
  float tuned_ms;         /* sweep time of the chosen shape */
} qtv_batch_info;

QTV_API int qtv_batch_plan(qtv_handle h, int n, const qtv_grid* grids, const void* const* psis,
                           const char* tune_cache, void* stream);
QTV_API int qtv_batch_info_get(qtv_handle h, qtv_batch_info* out);
QTV_API int qtv_batch_run(qtv_handle h, uint64_t* face_ids, int8_t* winding, uint64_t capacity,
                          uint64_t* offsets, float* xyz, float* resid, uint8_t* flags, int mode,
                          float fallback_resid, void* stream);

/*
 * Node form of the circulation (Sec. 2.2.2): for every node and each of the
 * three grid planes through it, the circulation of Eq. 5 around the ring of
 * the node's eight in-plane neighbours (the 2h x 2h square centred on the
 * node, counter-clockwise about the plane normal +z, +x, +y for the planes
 * xy, yz, zx), reported as the integer S = C / (2 pi) in [-3, 4] (|S| = 4
 * needs all eight edge differences at exact +-pi ties and reads 4).  A node is a
 * vortex node when max over its planes |C| > pi, i.e. some S != 0.  S = 0 where
 * the ring leaves the grid or passes through a NaN/Inf node (the centre node
 * is not on its ring).  Each ring edge uses the integer branch crossing of
 * qtv_identify, so S equals the sum of the four incident plaquette windings
 * whenever those are defined; it equals the FP64 definition on every ring
 * whose eight edge phase differences lie at least 1e-4 rad from +-pi.
 *
 *   psi       device, complex64 field (conventions above; 8-byte aligned).
 *   node_ids  device, uint64[capacity]: linear indices (k*ny + j)*nx + i of
 *             the vortex nodes, ascending.
 *   circ      device, int8[capacity][3]: S of the planes xy, yz, zx of each
 *             listed node.
 *   capacity  length of node_ids (and of circ in triples).
 *   count     device, one uint64: receives the number of vortex nodes; if it
 *             exceeds capacity the lists are incomplete (retry with a larger
 *             capacity).  capacity = 0 with NULL lists counts only.
 *   dense     device int8[3][nz][ny][nx] receiving S of every node and plane,
 *             or NULL.
 * The handle keeps its own workspace for this call (staging of capacity
 * records, per-(plane, band) tables); it grows on demand outside stream
 * capture.  Grids must have fewer than 2^52 nodes.
 */
QTV_API int qtv_node_circulation(qtv_handle h, const qtv_grid* grid, const void* psi,
                                 uint64_t* node_ids, int8_t* circ, uint64_t capacity,
                                 uint64_t* count, int8_t* dense, void* stream);

/*
 * The same node form (Sec. 2.2.2) from the pierced-face list of
 * qtv_identify instead of from psi: the ring of a node in a plane encloses
 * the four plaquettes of that plane at the node, its interior edges cancel,
 * so S is the sum of their windings.  Per node row one warp adds the
 * windings of the faces of the four neighbouring face rows and stages the
 * row's vortex nodes; a scan over the rows and a scatter list them.  Work is
 * per face, not per node.
 *
 *   face_ids, winding, n, n_dev  the ascending output of qtv_identify for
 *             this grid (n entries, or min(n, *n_dev) if n_dev is given).
 *   node_ids, circ, capacity, count  as qtv_node_circulation.
 *   tie       device uint32: non-zero when the outputs are not valid: 1 when
 *             a face has winding 2 (W mod 4 = 2: four exact +-pi ties), whose
 *             sign the face list does not carry (call qtv_node_circulation);
 *             2 if the staging buffer (sized for four nodes per face) ran
 *             out, which the sizing excludes.
 * Equal to qtv_node_circulation node for node when psi is finite (the
 * identification reported qtv_stats.nonfinite == 0: rings through a
 * non-finite node count 0 there, while the identification drops the faces
 * touching it) and tie stays 0.  Rows up to 4000 nodes; fewer than 2^32
 * faces; the handle keeps row tables of ny * nz entries and a staging buffer
 * of 4 n entries plus 8192 per resident warp.  QTV_ERR_STATE if they must
 * grow during stream capture.
 */
QTV_API int qtv_node_circulation_faces(qtv_handle h, const qtv_grid* grid,
                                       const uint64_t* face_ids, const int8_t* winding,
                                       uint64_t n, const uint64_t* n_dev, uint64_t* node_ids,
                                       int8_t* circ, uint64_t capacity, uint64_t* count,
                                       uint32_t* tie, void* stream);

/*
 * Density error of the sample points (Eq. 7, Sec. 5):
 *   e = (sum over the n points of |rho(p)|) / (n * rho_bar),
 * rho = |psi|^2 of the trilinearly interpolated field at p (Sec. 5: psi is
 * linearly interpolated between nodes), rho_bar = mean |psi|^2 over all nodes.
 *
 *   xyz    device float[n][3], positions origin + h * (grid coordinates), as
 *          written by qtv_localize.  A point outside the grid gets rho = NaN
 *          (and e becomes NaN).
 *   n      host bound on the number of points; n_dev (optional device uint64)
 *          limits it to min(n, *n_dev) without a host synchronisation.
 *   rho    optional device float[n]: rho at each point (FP32 interpolation).
 *   out    device double[3]: {e, mean |rho| over the points, rho_bar}; e = 0
 *          for no points.
 * Sums are FP32 over runs of at most 8 squares and FP64 across runs, in an
 * order fixed by the device's SM count, so repeated calls agree bit for bit.
 */
QTV_API int qtv_density_error(qtv_handle h, const qtv_grid* grid, const void* psi,
                              const float* xyz, uint64_t n, const uint64_t* n_dev, float* rho,
                              double* out, void* stream);

/*
 * Sample refinement (Sec. 3.3.3, "Locating more accurate sample points"): an
 * estimate x0 of a core sample (the paper starts from the box means of its
 * graph reduction; here any points, or the centres of pierced faces) moves to
 * a minimizer of the density rho = |psi|^2 (Eq. 6) within the plane through x0
 * perpendicular to the local core direction t, taken from the pseudo-vorticity
 * t = grad Re psi x grad Im psi at x0 (normalized).
 *
 *   psi between nodes is the trilinear interpolant; rho and grad rho are those
 *   of the interpolant within the cell floor(x).  grad Re psi and grad Im psi
 *   are central-difference node gradients (one-sided on the boundary)
 *   interpolated trilinearly.  Descent on the in-plane gradient g: each step
 *   starts at alpha = 2 rho / |g|^2 and halves alpha until
 *   rho(x - alpha g) <= rho(x) - 1e-4 alpha |g|^2 with the new point inside
 *   the grid and inside the box |x - x0|_inf <= 1 grid spacing (steps leaving
 *   either are rejected, not projected); it stops, converged, when no step of
 *   length >= tol grid spacings decreases rho that way, or after max_iter
 *   accepted steps.  FP32 arithmetic, positions carried relative to the cell
 *   of x0.
 *
 *   xyz0      device float[n][3] world positions (origin + h * grid coords),
 *             or NULL;
 *   face_ids  device uint64[n] face ids whose face centres are x0, or NULL;
 *             exactly one of the two is given.
 *   n, n_dev  host bound on the count; optional device uint64 limiting it to
 *             min(n, *n_dev) (to follow qtv_identify without a host sync).
 *   max_iter  step limit (200 in the tests); tol  step length in grid
 *             spacings below which the search stops (1e-7 in the tests).
 *   xyz       device float[n][3]: refined world positions (x0 when no
 *             tangent exists).
 *   rho       optional device float[n]: rho at the result (NaN for x0 outside
 *             the grid).
 *   tangent   optional device float[n][3]: t (0 when none).
 *   detj      optional device float[n]: determinant of the 2x2 real Jacobian
 *             of psi in an orthonormal in-plane basis at the result (the
 *             conditioning of the zero).
 *   iters     optional device int32[n]: accepted steps.
 *   flags     device uint8[n]: QTV_REFINE_* bits.
 */
#define QTV_REFINE_CONVERGED 1u
#define QTV_REFINE_NO_TANGENT 2u /* zero pseudo-vorticity or x0 outside the grid */
#define QTV_REFINE_MAX_ITER 4u
QTV_API int qtv_refine_samples(qtv_handle h, const qtv_grid* grid, const void* psi,
                               const float* xyz0, const uint64_t* face_ids, uint64_t n,
                               const uint64_t* n_dev, int max_iter, float tol, float* xyz,
                               float* rho, float* tangent, float* detj, int32_t* iters,
                               uint8_t* flags, void* stream);

/*
 * Sample graph over pierced faces (Sec. 3.1) and its connected components,
 * the independent lines of Sec. 3.2.  Two pierced faces are adjacent when
 * they bound the same unit cell (all eight corners in the grid): a core line
 * through a cell pierces the face it enters by and the face it leaves by,
 * and a cell with 4 or 6 pierced faces links all of them (a branch, as at a
 * reconnection).  A face has at most 10 neighbours.
 *
 *   face_ids  device uint64[n], strictly ascending (as from qtv_identify).
 *   n, n_dev  host bound on the count (< 2^32 - 1); optional device uint64
 *             limiting it to min(n, *n_dev).
 *   nbr       device uint32[n][10]: indices (into face_ids) of the
 *             neighbours, ascending, then 0xFFFFFFFF.
 *   deg       device uint8[n]: number of neighbours.
 *   comp      device uint32[n]: component label of each face = the lowest
 *             face index of its component (so components are numbered in
 *             the order of their lowest index, as a depth-first traversal
 *             from the lowest unvisited face finds them).
 *   ncomp     device uint64: number of components (QTV_COUNT_TIMEOUT if a
 *             bounded retry loop of the union-find gave up).
 * Entries beyond min(n, *n_dev) are not written.  The handle keeps a row
 * table of (ny * nz + 1) words.
 */
QTV_API int qtv_face_graph(qtv_handle h, const qtv_grid* grid, const uint64_t* face_ids, uint64_t n,
                           const uint64_t* n_dev, uint32_t* nbr, uint8_t* deg, uint32_t* comp,
                           uint64_t* ncomp, void* stream);

/*
 * The paper's own graph (Sec. 3.1) over vortex nodes: two vortex nodes are
 * adjacent when they are neighbours along a grid line (6-connectivity), and
 * its connected components (Sec. 3.2), as for qtv_face_graph.
 *
 *   node_ids  device uint64[n]: strictly ascending linear node indices (as
 *             from qtv_node_circulation).
 *   nbr       device uint32[n][6]: neighbour indices (into node_ids),
 *             ascending, then 0xFFFFFFFF; deg, comp, ncomp as in
 *             qtv_face_graph (components labelled by their lowest index).
 */
QTV_API int qtv_node_graph(qtv_handle h, const qtv_grid* grid, const uint64_t* node_ids, uint64_t n,
                           const uint64_t* n_dev, uint32_t* nbr, uint8_t* deg, uint32_t* comp,
                           uint64_t* ncomp, void* stream);

/*
 * Vortex-core lines of a sample graph (Sec. 3.4): classification, ordering,
 * orientation, and uniform Catmull-Rom curves, on the graph that
 * qtv_face_graph builds over pierced faces (the paper first thins its samples
 * by box means, Sec. 3.3.2; here the pieces run through every face sample).
 *
 * Classification of a component: Type III when a sample has more than two
 * neighbours (branch points, as at reconnections), Type II (a closed loop)
 * when every sample has exactly two and there is more than one, else Type I.
 * Pieces: a Type I component is one open piece from its lower end sample; a
 * Type II component is one closed piece from its lowest sample towards the
 * lower of that sample's neighbours; a Type III component splits at its
 * branch points into chains, each started at a branch point b through
 * neighbour v, from the branch side that comes first in (b, v) order (a chain
 * returning to b is closed; dead ends never start a chain).  A piece's
 * samples run along the circulation direction (Sec. 3.4, right-hand rule):
 * the piece is reversed when the sum over its segments of
 * (p[i+1] - p[i]) . d[i] is negative, d the sample's face normal times W (a
 * closed piece keeps its first sample).
 */
typedef struct {
  uint64_t first;     /* offset of the piece's samples in the node list */
  uint32_t count;     /* samples in the piece */
  uint32_t component; /* component label (lowest face index) */
  uint8_t closed;     /* 1: the last sample connects back to the first */
  uint8_t comp_type;  /* 1, 2, 3: Type I, II, III of the component */
  uint8_t reversed;   /* 1: flipped to follow the circulation direction */
  uint8_t reserved[5];
} qtv_piece;

/*
 *   n, n_dev     samples (faces) and an optional device bound on them.
 *   nbr, deg, comp  the outputs of qtv_face_graph.
 *   xyz          device float[n][3], the sample positions.
 *   face_ids, winding  device, the faces and W of the samples (orientation);
 *                both NULL: pieces keep their walk order.
 *   pieces       device qtv_piece[piece_cap], ordered by (start sample, first
 *                neighbour) of the walk that found them.
 *   nodes        device uint32[node_cap]: sample indices of all pieces, each
 *                piece a contiguous run (branch samples appear in every piece
 *                they end).
 *   counts       device uint64[2]: number of pieces and of node entries.  If
 *                either exceeds its capacity the outputs are incomplete;
 *                capacity 0 with NULL outputs counts only.
 */
QTV_API int qtv_line_pieces(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                            const uint8_t* deg, const uint32_t* comp, const float* xyz,
                            const uint64_t* face_ids, const int8_t* winding, qtv_piece* pieces,
                            uint64_t piece_cap, uint32_t* nodes, uint64_t node_cap,
                            uint64_t* counts, void* stream);

/*
 * Uniform Catmull-Rom curves through the samples of each piece (Sec. 3.4):
 * per_segment points on each segment between consecutive samples, the end
 * samples repeated as outer control points for open pieces and the samples
 * wrapped for closed ones, plus the last sample of an open piece (a piece of
 * one sample is that point).  FP32 points.
 *
 *   npieces, npieces_dev  piece count and an optional device bound on it.
 *   curve        device float[curve_cap][3]; curve_first device uint64[npieces]:
 *                each piece's first point; length device float[npieces]: the
 *                polyline length of each curve (closing segment included for
 *                closed pieces; FP32 segment lengths summed in FP64 in a
 *                fixed order).
 *   total        device uint64: number of curve points (outputs incomplete
 *                when it exceeds curve_cap).
 */
QTV_API int qtv_piece_curves(qtv_handle h, const float* xyz, const uint32_t* nodes,
                             const qtv_piece* pieces, uint64_t npieces,
                             const uint64_t* npieces_dev, int per_segment, float* curve,
                             uint64_t curve_cap, uint64_t* curve_first, float* length,
                             uint64_t* total, void* stream);

/*
 * Thinning of line pieces by arc length, a parallel reading of the box means
 * of Sec. 3.3.2 (which replace the samples inside a box of side d by their
 * mean, so that the box size sets the spacing of the final samples): the
 * samples of each ordered piece are grouped by the box index floor(s / box)
 * of their arc length s along the piece, and each group becomes its mean.
 * s sums the segment lengths (FP64, rounded to units of 2^-32 of the
 * position unit), so it is exact in any order; means are FP64 sums in sample
 * order, rounded to FP32.  The paper traverses the graph box by box instead,
 * which is sequential; the groups here never span two pieces.
 *
 *   xyz, nodes, pieces  the sample positions and the output of
 *                qtv_line_pieces (nnodes node entries, npieces pieces).
 *   box          box length, in the units of xyz.
 *   out_xyz      device float[out_cap][3]: the group means, piece by piece.
 *   out_pieces   device qtv_piece[npieces]: the pieces over out_xyz (first,
 *                count of the means; other fields copied).
 *   total        device uint64: number of means (outputs incomplete when it
 *                exceeds out_cap).
 * The means can be refined with qtv_refine_samples and drawn with
 * qtv_piece_curves (node list 0, 1, 2, ...).
 */
QTV_API int qtv_thin_pieces(qtv_handle h, const float* xyz, const uint32_t* nodes,
                            const qtv_piece* pieces, uint64_t npieces, uint64_t nnodes, float box,
                            float* out_xyz, uint64_t out_cap, qtv_piece* out_pieces,
                            uint64_t* total, void* stream);

/*
 * Box-mean reduction of a sample graph (Sec. 3.3.1-3.3.2), data-parallel:
 * the paper collapses, box by box along each line, the samples a box of side
 * d reaches into their mean, keeping the edges that leave the box, and
 * repeats whole passes until the samples settle.  Here each pass lays a
 * lattice of boxes of side `box` over space (shifted by box / 2 in every axis
 * on odd passes); the samples of one box that are connected through edges
 * inside it form a cluster, which becomes one node at the mean of its
 * members' positions with every edge leaving it.  Passes repeat until one pass
 * of each lattice merges nothing (a fixed point), at most max_passes.  The
 * result does not depend on the numbering of the samples: positions are held
 * in fixed point (integers in units of 2^-32 of the length unit: x 2^32
 * rounded to the nearest integer, ties to even), a mean is
 * floor((sum + floor(c / 2)) / c) over
 * the c members, and a cluster is named by the lowest input index it contains.
 *
 *   n, n_dev     host bound on the node count (< 2^32 - 1) and an optional
 *                device uint64 limiting it to min(n, *n_dev).
 *   nbr, deg     device uint32[n][stride] neighbour table (ascending, then
 *                0xFFFFFFFF) and uint8[n] degrees, as from qtv_face_graph
 *                (stride 10) or qtv_node_graph (stride 6).
 *   xyz          device float[n][3]: positions below 4096 in magnitude, in
 *                the unit of box (e.g. grid units); larger or non-finite
 *                values give unspecified clusters (memory stays in bounds).
 *   box          box side, 0 < box <= 32 (the paper takes d = k h, k in
 *                [3, 8]); max_passes in [1, 64] (the paper needs 2 to 5).
 *   label        device uint32[n]: the cluster of every node (its lowest
 *                node index), written.
 *   out_xyz      device double[n][3]: at every index r with label[r] == r
 *                the cluster's mean position (exact); other entries are
 *                scratch and unspecified.
 *   counts       device uint64[2]: clusters and passes made
 *                (QTV_COUNT_TIMEOUT as clusters if a bounded union-find
 *                retry loop gave up).
 * Asynchronous, capture-safe once the handle's workspace has reached n.
 */
QTV_API int qtv_box_reduce(qtv_handle h, uint64_t n, const uint64_t* n_dev, const uint32_t* nbr,
                           const uint8_t* deg, int stride, const float* xyz, float box,
                           int max_passes, uint32_t* label, double* out_xyz, uint64_t* counts,
                           void* stream);

/*
 * Kernel timing trace.  While enabled, the handle records a pair of CUDA
 * events on the launching stream around each of its kernel launches (names:
 * "sweep", "seg_scan", "scatter", "stats", "localize", "emit_pack", "batch"
 * for one replay of a batch graph, "encode", "network", "head" for the
 * parts of learned localization, "node_form", "node_scan", "node_scatter"
 * for the node form, "density" for the density error, "refine" for
 * sample refinement, "graph" for the face graph and its components, "lines"
 * and "curves" for line pieces and their curves, "thin" for their thinning,
 * "reduce" for the box-mean reduction).
 * qtv_trace_read waits for the recorded events, writes up to max_entries
 * per-kernel totals (launch count and summed device time) and, if reset is
 * nonzero, clears the record.  Tracing adds host work per launch and a gap
 * of about two microseconds per event on the device; leave it off outside
 * measurement.
 *
 * Calls are safe to capture into a CUDA graph (stream capture of the calling
 * stream) once their workspace exists: the library allocates and
 * synchronises nothing on the way, provided qtv_reserve (or one earlier call
 * of the same shape) has sized the workspace.  A traced launch inside a
 * capture becomes a pair of event-record nodes of the graph; the pair is
 * timed on each replay and qtv_trace_read gives the last replay's time
 * (read after the replay has finished; one record per captured launch).
 *
 * qtv_trace_filter restricts tracing to the launches of one kernel name
 * (one of the names above; NULL or "" traces all).  QTV_ERR_ARG for an
 * unknown name (the filter is left unchanged).
 */
typedef struct {
  char name[24];
  uint32_t launches;
  float total_ms;
} qtv_trace_entry;

QTV_API int qtv_trace_enable(qtv_handle h, int on);
QTV_API int qtv_trace_filter(qtv_handle h, const char* name);
QTV_API int qtv_trace_read(qtv_handle h, qtv_trace_entry* out, int max_entries, int* n_entries,
                           int reset);

#ifdef __cplusplus
}
#endif

#endif /* QTV_H */
