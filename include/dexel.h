/*
 * dexel.h -- C ABI of the GB300 dexel offset library (libdexel.so).
 *
 * Morphological offsets of a shape stored as a dexel buffer (Sec. 3.1, "Dexel
 * Representation"): a regular nx x ny grid of vertical rays; cell (i, j), centred at
 * ((i+1/2)h, (j+1/2)h), holds the sorted disjoint segments [z_in, z_out] where its ray is
 * inside the solid.  The library computes
 *   dilation   D_r(S) = { p : |p - x| <= r for some x in S }      (Sec. 3.1, dilation eq.)
 *   erosion    E_r(S) = complement of D_r(complement of S)         (Sec. 3.1, "Erosion")
 *   closing    E_r(D_r(S)),  opening  D_r(E_r(S))                  (Sec. 4, "Topological Cleaning")
 * exactly at the resolution of the input grid, by the two separable passes of Sec. 3.3:
 * an extrusion along x that keeps, for every z, the distance to the nearest parent column
 * (largest residual radius, Sec. 3.3 "3D Dilation"), then a dilation along y of those
 * pieces split into extruded rectangles and endpoint disks, the latter computed with
 * forward and backward half-space power diagrams of the endpoint seeds (Sec. 3.3
 * "2D Power Diagram", Eq. of power cells, App. B), and a per-column merge of the reached
 * intervals.  All work runs in CUDA kernels for sm_103a on one GPU.
 *
 * Layout (CSR, "col" numbers cells row-major: col = j*nx + i):
 *   col_off : int32[nx*ny + 1], col_off[0] = 0, non-decreasing; column col owns segments
 *             [col_off[col], col_off[col+1]).
 *   z       : pairs (z_in, z_out), float (DEXEL_FP32_PRED64) or double (DEXEL_FP64),
 *             2*nseg values; within a column z_in <= z_out < next z_in (strictly positive
 *             gaps; zero-length segments are allowed and denote a tangent sample).
 * The radius is given in grid spacings, k = r / h, so that the reach test
 * n = di^2 + dj^2 <= k^2 is exact on integers.  The output grid is the input grid (same
 * nx, ny, h); material pushed beyond the xy range of the grid is dropped, z is unbounded.
 * Columns outside the grid take part neither in S nor in its complement.
 *
 * Memory: every pointer in dexel_grid_in / dexel_grid_out and the workspace are DEVICE
 * pointers owned by the caller.  Inputs are never written.  Calls are ordered on the
 * given CUDA stream (a cudaStream_t passed as void*; NULL = legacy default stream); they
 * synchronise that stream internally to size intermediate buffers and return only after
 * the result is complete.  No exception or abort crosses this boundary: every failure is a
 * dexel_status.
 */
#ifndef DEXEL_H
#define DEXEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DEXEL_OK = 0,
  DEXEL_ERR_INVALID_ARG = -1, /* null pointer, bad size, k < 0 or not finite, h <= 0 ...  */
  DEXEL_ERR_BAD_CSR = -2,     /* offsets not monotone, z_in > z_out, gap <= 0, NaN        */
  DEXEL_ERR_CAPACITY = -3,    /* output or workspace too small; see dexel_last_required  */
  DEXEL_ERR_CUDA = -4,        /* a CUDA runtime call failed                                */
  DEXEL_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up                        */
  DEXEL_ERR_NOMEM = -6,       /* host-side allocation failed                               */
  DEXEL_ERR_NO_PLAN = -7      /* dexel_offset_enqueue: no plan recorded for this offset, or
                                 the data needed more than the plan (call dexel_dilate /
                                 dexel_erode, which plans again)                            */
} dexel_status;

/* Storage precision of the endpoints (input, intermediate and output).
 * DEXEL_FP64:        double endpoints, every computation in double.
 * DEXEL_FP32_PRED64: float endpoints; the power-diagram breakpoint and dominance
 *                    predicates and the merge comparisons are decided with double-accurate
 *                    arithmetic (an error-bounded float filter, double when undecided);
 *                    output endpoints are computed in double and rounded once to float. */
typedef enum { DEXEL_FP64 = 0, DEXEL_FP32_PRED64 = 1 } dexel_mode;

typedef enum { DEXEL_DILATE = 0, DEXEL_ERODE = 1, DEXEL_CLOSE = 2, DEXEL_OPEN = 3 } dexel_op;

/* Analytic primitives for dexel_raycast (world units; the grid's columns sit at
 * ((i + 1/2) h, (j + 1/2) h)). */
typedef enum { DEXEL_SPHERE = 0, DEXEL_BOX = 1, DEXEL_SHELL = 2 } dexel_prim_kind;
typedef struct {
  int32_t kind;  /* dexel_prim_kind */
  int32_t pad;
  double p[7];   /* sphere: cx cy cz R; box: x0 x1 y0 y1 z0 z1; shell (hollow sphere, outer
                    radius R, inner radius R - t): cx cy cz R t */
} dexel_prim;

/* Boolean operations of two grids (CSG in dexel space). */
typedef enum { DEXEL_UNION = 0, DEXEL_INTERSECT = 1, DEXEL_DIFFERENCE = 2 } dexel_bool_op;

typedef struct {
  int32_t nx, ny;         /* grid size, 1 <= nx, ny <= 32768                                */
  double h;               /* xy spacing, in the same units as z (> 0)                       */
  const int32_t* col_off; /* device, nx*ny + 1 entries                                      */
  const void* z;          /* device, 2*nseg endpoints (float or double, see dexel_mode)      */
  int64_t nseg;           /* number of segments (= col_off[nx*ny])                          */
} dexel_grid_in;

typedef struct {
  int32_t* col_off;     /* device, nx*ny + 1 entries, written                              */
  void* z;              /* device, room for 2*capacity_seg endpoints, written               */
  int64_t capacity_seg; /* size of z in segments                                           */
  int64_t nseg;         /* written on return: number of output segments (also when the
                           call fails with DEXEL_ERR_CAPACITY, so the caller can retry)    */
} dexel_grid_out;

typedef struct dexel_ctx dexel_ctx;

/* Create / destroy a context bound to CUDA device `device`.  The context owns only small
 * tables (the half-width table w[n] = h sqrt(k^2 - n), reach table) and status words, the
 * scratch it allocates when a call passes no workspace, and the plans (tapes) its
 * synchronous offsets recorded for dexel_offset_enqueue.  A context is not thread-safe: one
 * host thread at a time calls it (threads that need concurrent calls use a context each).
 *
 * Kernel choices are read from the environment when the context is created (for testing
 * and tuning; every choice gives the same result):
 *   DEXEL_PASS1=sweep|gather|lane   pass 1 as the per-row sweep, the per-column window
 *                                   kernel, or the lane-per-column window kernel at every
 *                                   reach (default: per-lane merges up to reach 2, the
 *                                   lane-per-column window kernel up to 128, the sweep beyond)
 *   DEXEL_PASS1_GW=1|2|4|8          warps a pass-1 tile (default by reach)
 *   DEXEL_PASS1_ECAP=256..16384     events a pass-1 tile holds (a power of two; default by
 *                                   density)
 *   DEXEL_PASS1_RING=0|1            pass 1 in one walk through per-lane ring regions (1,
 *                                   default) or in a counting and a writing walk
 *   DEXEL_PASS1_RING_CAP=16..1024   pieces a lane's ring region holds (default up to 256;
 *                                   a tile with a lane beyond it is walked again into place)
 *   DEXEL_PASS1_ECAP_RULE=mean|max  event room a tile by the mean density of the windows, the
 *                                   few denser columns redone by a second launch (mean,
 *                                   default), or room for the densest window from the start
 *   DEXEL_PASS1_ECAP_MUL=x          rule "mean": room for x times twice the mean window's
 *                                   events (0.5 .. 64).  Default (none of the three set):
 *                                   at reach >= 48 the room with the least window events per
 *                                   resident warp over the first launch and the redo launch,
 *                                   from a histogram of the tiles' window sizes; below, x = 1
 *   DEXEL_PASS1_BLOCK_CAP=1..3      the costed room counts at most this many blocks an SM
 *                                   (default 2: the 80-register plan of a third block spills
 *                                   about what it gains)
 *   DEXEL_PASS1_TILE_REDO=0|1       a tile whose window exceeds the room goes whole to the
 *                                   redo launch (1, default) or is split into narrower runs
 *                                   of columns (0)
 *   DEXEL_LEVEL_SLOTS=2..16         interval slots a lane of the pass-2 level walks holds in
 *                                   shared memory (default 8 below reach 48, 6 up to 64, 12
 *                                   beyond)
 *   DEXEL_LEVEL_SPILL=0..256        intervals a lane writes beyond its slots to its own
 *                                   region in global memory (default 64; a list longer than
 *                                   slots + spill is walked again straight into place)
 *   DEXEL_PASS1_NBUF=1|2            event buffers a pass-1 tile (2: every window that fits is
 *                                   merged from its sources' runs; 1: those of up to half the
 *                                   room, the others sorted; default 2 where it costs no block
 *                                   an SM)
 *   DEXEL_BLOCK_MB=n                split an offset into blocks of whole y lines when its
 *                                   S_mid, packed copy and level lists would take more than
 *                                   n MB (default: 0.45 of the device memory free when the
 *                                   context is created)
 *   DEXEL_PASS1_PRUNE=0|1           drop S_mid pieces whose capsule slice a neighbouring
 *                                   piece with a smaller dx contains at every level (1,
 *                                   default; the result is the same)
 *   DEXEL_PASS2=sweep|tiled         pass 2 as the per-line sweep or the tiled gather instead
 *                                   of the level unions
 *   DEXEL_LANE_GATHER_MAX=R         the pass-2 gather with one lane a column up to reach R
 *                                   (default 4)
 *   DEXEL_LEVELS_EXACT=0|1          level walks at reach >= 32 read S_mid itself (default 0)
 *   DEXEL_GATHER_BUCKET_MAX=256..8192  largest bucket (intervals a column, a power of two) the
 *                                   level gather grows to when many columns had to unite
 *                                   their bucket part way (default 512)
 *   DEXEL_BATCH_MAX_COLS=n          batched calls: shapes above n columns take the
 *                                   single-shape path (default 131072) */
dexel_status dexel_ctx_create(dexel_ctx** ctx, int device);
void dexel_ctx_destroy(dexel_ctx* ctx);

/* Suggested workspace size in bytes for an offset of `in` by k spacings.  The true need is
 * data dependent (intermediate pieces grow with k, Sec. 3.4); when a call finds the
 * workspace too small it returns DEXEL_ERR_CAPACITY and dexel_last_required() gives the
 * size that suffices.  Never returns less than the fixed part. */
size_t dexel_workspace_size(const dexel_grid_in* in, double k, dexel_mode mode);

/* Bytes of workspace the last call on ctx needed (valid after DEXEL_ERR_CAPACITY too). */
size_t dexel_last_required(const dexel_ctx* ctx);

/* Check a CSR grid on the device: offsets start at 0, are non-decreasing and end at nseg;
 * every segment has z_in <= z_out, consecutive segments of a column have z_out < next
 * z_in, no NaN.  Returns DEXEL_OK or DEXEL_ERR_BAD_CSR. */
dexel_status dexel_validate(dexel_ctx* ctx, const dexel_grid_in* in, dexel_mode mode,
                            void* ws, size_t ws_bytes, void* stream);

/* Dilation of `in` by a ball of radius k*h (Sec. 3.1 dilation eq., Sec. 3.3 two passes).
 * k >= 0 and finite.  On success out->col_off / out->z hold the result and out->nseg its
 * size.  If out->capacity_seg is too small: DEXEL_ERR_CAPACITY, out->nseg = required
 * size, out->z untouched.  If the workspace is too small: DEXEL_ERR_CAPACITY and
 * dexel_last_required(ctx) > ws_bytes. */
dexel_status dexel_dilate(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_mode mode,
                          dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream);

/* Erosion by a ball of radius k*h: the complement of the dilation of the complement
 * (Sec. 3.1 "Erosion"), with the complement taken per column on the fly (+-inf sentinels)
 * and undone when storing; results of zero length are dropped.  Same contract as
 * dexel_dilate. */
dexel_status dexel_erode(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_mode mode,
                         dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream);

/* Stream-ordered offset: dexel_dilate (op DEXEL_DILATE) or dexel_erode (DEXEL_ERODE) that
 * issues no host synchronisation, so that a caller can queue it behind its own work (or
 * between other kernels of one stream) without a round trip to the host.  It is not in the
 * paper; the two passes it runs are those of dexel_dilate.
 *   A synchronous dexel_dilate / dexel_erode on the same context records, for its element
 *   type, grid size (nx, ny), k and op, the counters it read at its synchronisations (its
 *   plan).  This call replays that plan: it enqueues the same kernels on `stream`, makes
 *   every redo launch (a redo finds nothing to do when the first launch finished), and
 *   returns without waiting.  Without a recorded plan it returns DEXEL_ERR_NO_PLAN and does
 *   nothing.  Plans whose synchronous call took a fallback fed with host-read data (the
 *   per-row sweeps, the tiled gather) are not recorded.
 *   ws must be a caller workspace (no allocation happens); out->capacity_seg bounds the
 *   output; out->nseg is set to -1.
 *   d_result : DEVICE int64[2] (caller-owned), written in stream order when the call returns
 *   DEXEL_OK: [0] DEXEL_OK, DEXEL_ERR_BAD_CSR, DEXEL_ERR_CAPACITY (output beyond
 *   capacity_seg or int32 offsets; [1] is then the size needed) or DEXEL_ERR_NO_PLAN (the
 *   data needed more room or another path than the plan: call dexel_dilate / dexel_erode);
 *   [1] the output's segment count.  out->z is written only when [0] is DEXEL_OK (out->col_off
 *   always).  A host-side failure (a bad argument, a workspace below the plan's need:
 *   DEXEL_ERR_CAPACITY with dexel_last_required) returns before anything is queued.  Any
 *   return other than DEXEL_OK leaves d_result unwritten: the call counts as not made (a
 *   DEXEL_ERR_NO_PLAN from a plan the context's state no longer matches may follow kernels
 *   already queued on the stream; they only touch the workspace and out->col_off). */
dexel_status dexel_offset_enqueue(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_op op,
                                  dexel_mode mode, dexel_grid_out* out, void* ws,
                                  size_t ws_bytes, void* stream, int64_t* d_result);

/* Closing (erode after dilate) or opening (dilate after erode) by the same radius; the
 * intermediate grid lives in the workspace.  op must be DEXEL_CLOSE or DEXEL_OPEN. */
dexel_status dexel_morph(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_op op,
                         dexel_mode mode, dexel_grid_out* out, void* ws, size_t ws_bytes,
                         void* stream);

/* 2D offsets of dexel images (Sec. 3.2, "Half-Space Voronoi Diagram of Segments and 2D
 * Offsets": a 2D shape given as parallel segments on a regular grid, dilated by a disk), for
 * every row of the grid at once: row j (the nx columns with this j) is an independent 2D image
 * in its (x, z) plane -- a slice of a CT stack, a layer of a print -- offset by a disk of
 * radius k*h (k in spacings, as for dexel_dilate).  op: DEXEL_DILATE, or DEXEL_ERODE (the
 * complement of the dilation of the complement, within each row).  Pass 1 (the extrusion
 * along x) is the 3D one; the y pass keeps, for every column, its own pieces' slices
 * [a - w, b + w], w = h sqrt(k^2 - dx^2).  Same layout, workspace and retry contract as
 * dexel_dilate (k at most 1024; DEXEL_ERR_CAPACITY when a column's union outgrows every
 * gather bucket). */
dexel_status dexel_offset_slices(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_op op,
                                 dexel_mode mode, dexel_grid_out* out, void* ws, size_t ws_bytes,
                                 void* stream);

/* Ray casting of analytic primitives into a dexel grid (Sec. 1: implicit shapes turn into
 * ray representations directly, without meshing; Sec. 3.1 "Dexel Representation").  Column
 * (i, j) of the nx x ny grid of spacing h casts the vertical ray through ((i+1/2)h,
 * (j+1/2)h): a sphere gives the chord cz -+ sqrt(R^2 - d^2) where d^2 < R^2, a box [z0, z1]
 * where x0 < x < x1 and y0 < y < y1, a hollow sphere the sphere's chord minus the inner
 * sphere's open chord; tangent rays give nothing.  The chords of a column are united (closed
 * union); FP32 mode rounds the united ends to the nearest float and joins segments that then
 * touch.  The heights are computed with correctly rounded double operations, one at a time.
 *   prims : DEVICE array of nprim primitives (caller-owned).
 *   out   : as for dexel_dilate; out->nseg = -1 with DEXEL_ERR_CAPACITY when a column is hit by
 *           more than 160 chords (not an output-size problem). */
dexel_status dexel_raycast(dexel_ctx* ctx, const dexel_prim* prims, int32_t nprim, int32_t nx,
                           int32_t ny, double h, dexel_mode mode, dexel_grid_out* out, void* ws,
                           size_t ws_bytes, void* stream);

/* The same with rays along axis 0 (x), 1 (y) or 2 (z, as dexel_raycast): the grid then spans
 * the other two axes in cyclic order -- x rays: columns over (y, z), heights are x; y rays:
 * columns over (z, x), heights are y -- so that the three views of one solid form a layered
 * depth image (three dexel sets, one an axis; Sec. 5, future work). */
dexel_status dexel_raycast_axis(dexel_ctx* ctx, const dexel_prim* prims, int32_t nprim,
                                int32_t axis, int32_t nx, int32_t ny, double h, dexel_mode mode,
                                dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream);

/* Offset of a three-view layered depth image (Sec. 5: "directly work on a LDI offset, i.e.
 * representing the shape with 3 dexel representations, one for each axis"; Sec. 4 notes the
 * threefold cost).  views[0..2] are the dexel sets of one solid along z, x and y (as made by
 * dexel_raycast_axis with axis 2, 0, 1), all with the same spacing h; the ball is isotropic,
 * so each view is offset on its own by the two-pass method: outs[v] receives
 * op(views[v]) for op in DEXEL_DILATE / ERODE / CLOSE / OPEN.  Host arrays of 3 entries with
 * device buffers; each output follows dexel_dilate's contract (outs[v].nseg the need on
 * DEXEL_ERR_CAPACITY).  Returns the first failing status.  Stats sum over the views. */
dexel_status dexel_offset_ldi(dexel_ctx* ctx, const dexel_grid_in* views, double k, dexel_op op,
                              dexel_mode mode, dexel_grid_out* outs, void* ws, size_t ws_bytes,
                              void* stream);

/* Boolean operation of two grids of the same size (CSG carried out in dexel space, Sec. 2
 * "(3)": the rays of a column combine on their own), column by column:
 *   DEXEL_UNION       closed union of a and b (touching segments join; an isolated
 *                     zero-length segment stays);
 *   DEXEL_INTERSECT   closed intersection; results of zero length are dropped;
 *   DEXEL_DIFFERENCE  the closure of a minus b (b's segments remove their open interiors);
 *                     results of zero length are dropped.
 * a, b: device CSR grids with the same nx, ny (h is taken from a) and the precision `mode`;
 * both are validated (DEXEL_ERR_BAD_CSR).  No arithmetic touches the heights: every output
 * end is an input end, in either precision.  Output, workspace and retry contract as for
 * dexel_dilate (ws may be NULL: library-owned scratch of 24 bytes a column). */
dexel_status dexel_boolean(dexel_ctx* ctx, dexel_bool_op op, const dexel_grid_in* a,
                           const dexel_grid_in* b, dexel_mode mode, dexel_grid_out* out, void* ws,
                           size_t ws_bytes, void* stream);

/* Thick shell of controllable thickness: the Boolean difference of the dilation and the
 * erosion by a ball of radius k*h (Sec. 4 "3D Printing"; the teaser figure's shell).  The two
 * offsets live in context-owned buffers; same contract as dexel_dilate. */
dexel_status dexel_shell(dexel_ctx* ctx, const dexel_grid_in* in, double k, dexel_mode mode,
                         dexel_grid_out* out, void* ws, size_t ws_bytes, void* stream);

/* Batched offsets: nshapes independent grids, each with its own radius and operation
 * (Sec. 3.3 applied to a table of shapes; no counterpart in the paper, which offsets one
 * model at a time).  ins / k / ops / outs are HOST arrays of nshapes entries whose grid
 * pointers are device pointers; outs[s].nseg receives each shape's segment count (the
 * needed count when its status is DEXEL_ERR_CAPACITY).  All shapes run together: one
 * grid-strided launch per stage over the table of every shape's tiles (validation, tables,
 * pass 1 with dominance pruning, packing, level unions, gather, count, scan, totals, write).
 * A closing / opening runs as two such sequences (its intermediate grid in engine memory,
 * sized from the last call of the same shapes).  The sequence is recorded as a CUDA graph
 * and replayed, through the output write, when the next call has the same shapes (sizes,
 * radii, operations): such a call synchronises the host once a sequence, to read the status
 * words.  Tile shapes are autotuned on the first call of a signature (see
 * dexel_set_batch_autotune).  Shapes of more than 131072 columns (environment
 * DEXEL_BATCH_MAX_COLS at context creation) take the single-shape path, one call each.
 * Scratch is library-owned (ws is used only by shapes on the single-shape path: the large
 * ones, reach above 127 spacings, or a window beyond the batch kernels' limits).  d_status
 * (device, nshapes int32, may be NULL) receives each shape's dexel_status.  Returns the
 * first failing status (or DEXEL_OK); DEXEL_ERR_INVALID_ARG when any argument is invalid
 * (nothing runs).  Synchronises the stream before returning. */
dexel_status dexel_offset_batched(dexel_ctx* ctx, int nshapes, const dexel_grid_in* ins,
                                  const double* k, const dexel_op* ops, dexel_mode mode,
                                  dexel_grid_out* outs, void* ws, size_t ws_bytes,
                                  int32_t* d_status, void* stream);

/* Turn the tile autotuning of dexel_offset_batched on (default) or off. */
void dexel_set_batch_autotune(dexel_ctx* ctx, int on);

/* Allocation-free dilation or erosion for small grids (the paper has no counterpart; this is
 * a deployment variant).  For callers that cannot allocate device memory when they need an
 * offset -- an application whose own pool owns the GPU's memory, a real-time loop that must
 * not pay cudaMalloc's implicit synchronisation, code running where allocation is
 * forbidden.  It runs the per-line sweep kernels of dexel_dilate / dexel_erode, but every
 * byte of scratch comes from one static 128 MiB device array inside the library; nothing is
 * allocated or freed (no ctx either).  The array is committed when the library's module is
 * loaded on a device (eagerly, or on first use under lazy loading) and is held by every GPU
 * that loads it until the process exits; a failure to load it is reported as DEXEL_ERR_CUDA.
 *   in, out : as for dexel_dilate (device buffers owned by the caller).
 *   op      : DEXEL_DILATE or DEXEL_ERODE.
 * out->nseg on return:
 *   >= 0 and <= capacity_seg   success (DEXEL_OK): the number of output segments;
 *   > capacity_seg             DEXEL_ERR_CAPACITY: the caller's output is too small, nseg is
 *                              the size it needs (retry with a larger buffer);
 *   -1                         DEXEL_ERR_CAPACITY: the grid is beyond the static scratch
 *                              (nx*ny > 65536, k > 32, or data needing more scratch than the
 *                              array holds); retrying cannot help.
 * The array serves unions of a few spheres or boxes up to 256 x 256 columns at k = 32 (about
 * 25 MB of intermediate pieces there); dense stacks of segments need more and are refused.
 * On DEXEL_ERR_CAPACITY out->z is not written; with nseg = -1 out->col_off is not written
 * either.
 * Every call looks up the array's device address in the current device's context
 * (cudaGetSymbolAddress) and reads status words back with synchronous copies, so the call
 * synchronises `stream` several times and must not be made while `stream` (or a stream it
 * joins) is being captured into a CUDA graph.  All calls share the array and the next call
 * overwrites what the last one left: calls that overlap on the GPU (other streams or
 * threads) race. */
dexel_status dexel_offset_noalloc(const dexel_grid_in* in, double k, dexel_op op, dexel_mode mode,
                                  dexel_grid_out* out, void* stream);

/* Static description of a status code. */
const char* dexel_status_string(dexel_status s);

/* Device status bits after the last pass-2 level step (diagnostics; 16: a level list beyond
 * its buffer, the tiled gather took over; 32: a self-check found an index out of range). */
int dexel_last_levels_status(const dexel_ctx* ctx);

/* Detail of the last DEXEL_ERR_CUDA / DEXEL_ERR_NOMEM of the calling thread: the CUDA error
 * code and name and the library source line ("" when none). */
const char* dexel_last_error_detail(void);

/* Kernel launches issued by the last call on ctx (for launch accounting). */
int64_t dexel_last_launches(const dexel_ctx* ctx);

/* Turn per-stage timing on or off (off by default).  When on, each call brackets its
 * stages with CUDA events on the call's stream; dexel_last_stage_ms then reports the
 * device time of each stage of the last call (summed over both offsets of a closing or
 * opening): [0] validation + tables, [1] pass 1 (x extrusion), [2] pass 2 (y dilation with
 * per-piece radius: the gather kernels, or the sweep; the float copy of S_mid made before
 * the gather is in no stage), [3] output count + scan, [4] output write.  Returns the number
 * of entries written (at most max). */
void dexel_set_profiling(dexel_ctx* ctx, int on);
int dexel_last_stage_ms(const dexel_ctx* ctx, double* ms, int max);

/* With profiling on, the device time of single kernels of the last call, each bracketed by
 * its own CUDA events on the call's stream (0 when the kernel did not run): [0] the pass-1
 * window kernel (one lane per output column), [1] k_levels (per-source level unions of
 * pass 2), [2] k_lgather (their per-column union), [3] the packed float copy of S_mid (scan
 * + pack).  Summed over both offsets of a closing or opening.  Returns the number of entries
 * written (at most max, 4 in all). */
int dexel_last_kernel_ms(const dexel_ctx* ctx, double* ms, int max);

/* Sizes seen by the last call (summed over both offsets of a closing or opening):
 * [0] input segments, [1] S_mid pieces (pass-1 output), [2] pass-2 intervals before the final
 * complement/rounding, [3] output segments, [4] max pieces in one S_mid column, [5] window
 * gather: output columns redone by the shared-memory fallback kernel; per-line sweep: max
 * live elements in one sweep state, [6] device status bits of the last attempt (1: a per-warp
 * state array overflowed, 2: an arena overflowed, 4: malformed CSR, 8: output beyond int32
 * offsets), [7] attempts the last offset needed (the library grows its scratch and retries
 * when it owns the workspace), [8] second launches of the pass-1 window kernel for columns
 * whose window outgrew the first launch's event room, [9] blocks of y lines the offset ran in
 * (S_mid and the level lists exist for one block at a time; 1: the whole grid at once),
 * [10] pass-1 tiles walked twice because a lane outgrew its ring region, [11] output columns
 * whose level lists outgrew the gather's bucket (united straight from the lists), [12] that
 * bucket's size in intervals, [13] the event room of a pass-1 tile, [14] level lists of pass
 * 2 longer than a lane's slots (walked again straight into place).  Returns the number of
 * entries written (at most max, 15 in all). */
int dexel_last_stats(const dexel_ctx* ctx, int64_t* stats, int max);

/* Diagnostic counters of the last call: clock cycles per phase of the y sweep and mean
 * state sizes, filled only by builds compiled with -DDEXEL_PHASES (zero otherwise).
 * Returns the number of entries written (at most max, 16 in all). */
int dexel_last_phases(const dexel_ctx* ctx, uint64_t* ph, int max);

#ifdef __cplusplus
}
#endif

#endif /* DEXEL_H */
