/*
 * simplexenc.h -- C ABI of the GB300 (sm_103a) simplex-grid hash encoding library.
 *
 * The library computes the multiresolution simplex-lattice hash encoding of
 * Wen & Yang, "Efficient Encoding of Graphics Primitives with Simplex-based
 * Structures" (arXiv 2311.15439), its backward pass, the tiny fully connected
 * network that consumes it, the L2 loss of the image-fitting task and the Adam
 * update that trains tables and network, plus the 2^d multilinear hash-grid
 * encoder that the paper compares against.
 *
 * Conventions for every entry point:
 *   - Every buffer argument is a DEVICE pointer owned by the caller unless its
 *     comment says "host".  The library never allocates device memory and never
 *     frees caller memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  All device work is enqueued asynchronously on that stream; the
 *     call returns without synchronising.
 *   - Arguments are validated on the host before anything is enqueued.  A bad
 *     argument returns SXE_EINVAL (or SXE_EUNSUPPORTED for a valid but
 *     unimplemented combination) and enqueues nothing.  A CUDA launch error
 *     returns SXE_ECUDA.  No call aborts the process.  sxe_last_error() gives a
 *     message for the last failing call on the calling thread.
 *   - Gradient outputs accumulate (+=); the caller zeroes them when needed.
 *   - Layouts are row-major with the last index fastest.
 *   - Dimensions d = 2..5 are supported (the paper's n, Sec. 6.3 studies up to 7).
 *   - Points are meant to lie in [0,1]^d (Sec. 4.2 footnote).  Points outside
 *     it are still encoded (their lattice vertices hash like any other) as long
 *     as every scaled, skewed coordinate stays below 2^31 in magnitude; NaN
 *     input gives unspecified output but never an out-of-bounds access.
 */
#ifndef SIMPLEXENC_H
#define SIMPLEXENC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SXE_OK = 0,
  SXE_EINVAL = -1,        /* an argument is out of range or NULL where required */
  SXE_EUNSUPPORTED = -2,  /* valid but not implemented (e.g. d = 7)            */
  SXE_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed        */
  SXE_ENOMEM = -4         /* a caller-provided workspace or buffer is too small,
                             or the host could not allocate (serving requests)  */
} sxe_status;

typedef enum { SXE_SIMPLEX = 0, SXE_GRID = 1 } sxe_kind;
typedef enum { SXE_F32 = 0, SXE_F16 = 1, SXE_BF16 = 2 } sxe_dtype;
typedef enum { SXE_RES_RAW = 0, SXE_RES_EQUAL_MEM = 1 } sxe_res_mode;
typedef enum { SXE_INDEX_HASH = 0, SXE_INDEX_DENSE_COARSE = 1 } sxe_index_mode;

#define SXE_MAX_LEVELS 32

/*
 * Encoding description (Sec. 5, Sec. 5.1, Sec. 5.2).
 *   d            input dimension n of the paper, 2..5
 *   n_levels     L, 1..SXE_MAX_LEVELS
 *   n_features   F features per table entry: 1, 2, 4 or 8
 *   log2_T       table size T = 2^log2_T entries per level, 4..26
 *   base_res     resolution of level 0; level l has N_l = floor(base_res * growth^l)
 *   growth       per-level growth factor (>= 1)
 *   kind         SXE_SIMPLEX (the paper's method, n+1 vertices per level) or
 *                SXE_GRID (the 2^n-corner multilinear comparator, Algorithm 1)
 *   res_mode     SXE_RES_RAW, or SXE_RES_EQUAL_MEM to multiply N_l by
 *                (n+1)^((n-1)/(2n)) as Sec. 5.2 does for equal-memory comparisons
 *                (simplex only)
 *   table_dtype  storage type of the feature tables read by the forward pass
 *   out_dtype    type of the encoded output
 *   index_mode   SXE_INDEX_HASH: every level hashes its vertices (Sec. 5 a).
 *                SXE_INDEX_DENSE_COARSE: a level whose lattice box fits the table
 *                stores vertex v directly at sum_i v_i B^i (uint32, modulo T), where
 *                B = floor(top (1 + 2^-20)) + 2 coordinates per axis, top = s_l sqrt(n+1)
 *                (simplex) or N_l (grid), if B^n <= T; the other levels hash.  No
 *                collisions on those levels for points in [0,1]^n.
 */
typedef struct {
  int32_t d;
  int32_t n_levels;
  int32_t n_features;
  int32_t log2_T;
  double base_res;
  double growth;
  int32_t kind;
  int32_t res_mode;
  int32_t table_dtype;
  int32_t out_dtype;
  int32_t index_mode;
} sxe_encoding_desc;

typedef struct sxe_encoder sxe_encoder;  /* opaque: level constants only, no device memory */

/* Validates `desc` and computes the per-level constants on the host (Sec. 5.1):
 * the input multiplier N_l * m / sqrt(n+1) for the simplex (m = 1 or the Sec. 5.2
 * factor) or N_l for the grid, in FP64 rounded once to binary32, and the skew
 * factor F_n = (sqrt(n+1)-1)/n of Eq. 2.  *out receives a handle the caller
 * releases with sxe_encoder_destroy.  Thread-safe; the handle is immutable. */
sxe_status sxe_encoder_create(const sxe_encoding_desc* desc, sxe_encoder** out);
sxe_status sxe_encoder_destroy(sxe_encoder* enc);

/* Copies the binary32 per-level multipliers (host float[L]) and the integer level
 * resolutions N_l (host int32[L]) into caller arrays; either may be NULL. */
sxe_status sxe_encoder_level_params(const sxe_encoder* enc, float* level_scale, int32_t* level_res);

/* Copies the per-level box width B of the directly indexed levels into host int32[L]
 * (0 for a hashed level; all 0 under SXE_INDEX_HASH). */
sxe_status sxe_encoder_level_index(const sxe_encoder* enc, int32_t* box_width);

/* Backward strategy for the levels that are not summed in shared memory (sxe_encode_bwd,
 * sxe_encode_bwd_levels).  on = 0 (default): one thread per (point, level), every term added
 * to its table entry with its own reduction.  on = 1: a warp takes 32 consecutive points of one
 * level, finds the lanes whose vertices share a table entry (Sec. 5 step (e) adds all of them
 * into the same H_l[slot]) and adds each group's sum with one reduction; this pays when
 * consecutive points are spatially coherent (the samples along a ray, Sec. 6.2), where
 * neighbours share vertices.  The sums are the same up to floating-point reassociation.
 * SXE_EINVAL for a NULL encoder or on not 0 or 1.  Not thread-safe with concurrent calls on the
 * same encoder. */
sxe_status sxe_encoder_set_bwd_aggregation(sxe_encoder* enc, int32_t on);

/* Work-item order of the forward encoding (sxe_encode_fwd, sxe_encode_fwd_marked).  The
 * outputs are the same bit for bit in every order (each (point, level) item computes alone);
 * only the memory traffic differs.  SXE_FWD_ORDER_POINT_MAJOR: consecutive threads take the
 * levels of one point, then the next point, so every level's table is read at the same time.
 * SXE_FWD_ORDER_LEVEL_MAJOR: blocks take consecutive points of one level, the levels in turn, so
 * one or two levels' tables are read at a time; where all the tables exceed L2 but one level's
 * fits, a table sector fetched for one point stays in L2 for the later points of its level.
 * SXE_FWD_ORDER_AUTO (the default): level-major when L tables of T entries exceed the device's
 * L2 and one of them takes at most half of it, else point-major.  SXE_EINVAL for a NULL
 * encoder or another value.  Not thread-safe with concurrent calls on the same encoder. */
#define SXE_FWD_ORDER_AUTO 0
#define SXE_FWD_ORDER_POINT_MAJOR 1
#define SXE_FWD_ORDER_LEVEL_MAJOR 2
sxe_status sxe_encoder_set_fwd_order(sxe_encoder* enc, int32_t order);

/* Forward encoding, Sec. 5 steps (a)-(d): for every point and level, scale and skew
 * (Eq. 2) the point, find its simplex by sorting the fractional parts (Sec. 4.2),
 * weight its n+1 vertices barycentrically (Sec. 4.3), hash each vertex into that
 * level's table and interpolate; levels are concatenated.
 *   x       [n_points][d] binary32
 *   tables  [L][T][F] of desc.table_dtype
 *   out     [n_points][L*F] of desc.out_dtype (fully overwritten)
 * n_points may be 0 (nothing is enqueued).  The binary32 scale and skew use one
 * rounding per operation in a fixed order (p_i = x_i*s, sigma = sum left to right,
 * t = F_n*sigma, q_i = p_i + t); ties between equal fractional parts list the
 * lower axis first. */
sxe_status sxe_encode_fwd(const sxe_encoder* enc, const float* x, int64_t n_points,
                          const void* tables, void* out, void* stream);

/* sxe_encode_fwd that also sets, in the bitmap `touched` (L*T bits, the layout of
 * sxe_encode_bwd's), the bit of every table entry it reads: for the same points these are exactly
 * the entries whose gradient the backward pass adds to (Sec. 5 step (e) scatters into the entries
 * step (b) looked up), so a training step can mark them here and call the backward with touched =
 * NULL.  Bits are only set, never cleared.  Same arguments and errors as sxe_encode_fwd, plus
 * SXE_EINVAL for a NULL touched when n_points > 0. */
sxe_status sxe_encode_fwd_marked(const sxe_encoder* enc, const float* x, int64_t n_points,
                                 const void* tables, void* out, uint32_t* touched, void* stream);

/* Backward encoding, Sec. 5 step (e): for every point, level, vertex k and feature f,
 *   grad[(l*T + slot_k) * grad_stride + f] += w_k * dout[p][l*F + f]
 * with the same vertices and weights as the forward pass (recomputed).
 *   dout         [n_points][L*F] binary32
 *   grad         binary32 gradient storage; entry (l, slot) starts at float index
 *                (l*T + slot) * grad_stride.  grad_stride = F gives a dense [L][T][F]
 *                array; larger strides let the gradient live inside an
 *                interleaved optimiser-state record.  grad_stride must be a
 *                multiple of F and the byte address of every entry a multiple of
 *                4*F bytes (for F <= 4) or 16 bytes (F = 8).
 *   touched      optional bitmap of L*T bits (uint32 words, bit e%32 of word e/32
 *                for entry e = l*T + slot); every entry that receives a term gets
 *                its bit set.  NULL disables marking.
 * Accumulation order is unspecified (atomic adds), so results agree with the
 * exact sum to within floating-point reassociation.  Levels whose lattice box is
 * small are summed per thread block in shared memory first and added once per
 * block (see sxe_encode_bwd_kernel_count); one or two kernels on `stream`. */
sxe_status sxe_encode_bwd(const sxe_encoder* enc, const float* x, int64_t n_points,
                          const float* dout, float* grad, int64_t grad_stride,
                          uint32_t* touched, void* stream);

/* sxe_encode_bwd restricted to the levels [level_begin, level_end) (0 <= level_begin <=
 * level_end <= L; an empty range does nothing): only the terms of those levels are added and
 * only their entries are marked in `touched`.  Entries of different levels never share a
 * gradient address or a bitmap word when T >= 32, so a caller can run the optimiser on the
 * entries of one range (see sxe_step_touched on a sub-range of the state) while the backward
 * of another range runs on a second stream.  Same arguments and errors as sxe_encode_bwd,
 * plus SXE_EINVAL for a range outside [0, L]. */
sxe_status sxe_encode_bwd_levels(const sxe_encoder* enc, const float* x, int64_t n_points,
                                 const float* dout, float* grad, int64_t grad_stride,
                                 uint32_t* touched, int32_t level_begin, int32_t level_end,
                                 void* stream);

/* Number of kernels sxe_encode_bwd launches for n_points (1 or 2; 0 for none): levels
 * whose lattice box is small are first summed per thread block in shared memory and
 * added to the table once per block (many contributions per vertex would otherwise
 * serialise on the same addresses); the other levels take the direct path. */
int32_t sxe_encode_bwd_kernel_count(const sxe_encoder* enc, int64_t n_points);
/* The same for sxe_encode_bwd_levels on [level_begin, level_end) (0 for an empty or invalid range). */
int32_t sxe_encode_bwd_levels_kernel_count(const sxe_encoder* enc, int64_t n_points, int32_t level_begin,
                                           int32_t level_end);
/* Number of leading levels (0 <= n <= L) that sxe_encode_bwd sums per thread block in shared
 * memory for n_points points; they run as their own kernel, so a caller may run the levels
 * [0, n) and [n, L) through sxe_encode_bwd_levels on two streams at once (they share no
 * gradient address, nor a bitmap word when T >= 32).  Returns 0 for a NULL encoder or
 * n_points <= 0. */
int32_t sxe_encode_bwd_coarse_levels(const sxe_encoder* enc, int64_t n_points);

/* Gradient with respect to the points (the chain rule through Sec. 4.3's weights, Eq. 2's
 * skew and the level scale; the paper does not state it):
 *   dx[p][i] += sum_{l,f} dout[p][l*F+f] * d out[p][l*F+f] / d x_i
 * Simplex: inside the point's simplex the output is affine in the fractional parts q - c,
 * and d out / d q_i = H(v_{k+1}) - H(v_k) for the axis i added between vertices k and k+1
 * (Remark 2); d/dx = s_l (I + F_n 1 1^T) d/dq.  Grid: the derivative of the n-linear
 * weights, times N_l.  On faces and ties the value is the one-sided derivative of the
 * simplex (cell) the forward pass picks.
 *   tables  [L][T][F] of the encoder's table dtype (dense, as sxe_encode_fwd)
 *   dout    [n_points][L*F] binary32
 *   dx      [n_points][d] binary32, accumulated (+=); zero it for a plain gradient.
 * All device pointers, caller-owned, 4-byte aligned (tables as sxe_encode_fwd).
 * One kernel on `stream`. */
sxe_status sxe_encode_bwd_input(const sxe_encoder* enc, const float* x, int64_t n_points,
                                const void* tables, const float* dout, float* dx, void* stream);

/* The lattice vertices the encoding reads, for testing and inspection:
 *   slots    [n_points][L][V] uint32 table slots (0..T-1) of each vertex
 *   weights  [n_points][L][V] binary32 interpolation weights
 * with V = d+1 (simplex, in the walk order of Sec. 4.2: base vertex first) or
 * V = 2^d (grid, corner b at index sum_i b_i 2^(d-1-i)).  Either pointer may be NULL. */
sxe_status sxe_encode_vertices(const sxe_encoder* enc, const float* x, int64_t n_points,
                               uint32_t* slots, float* weights, void* stream);

/* Plain binary32 comparator of the simplex encoding: one thread per point loops over
 * the levels, orders the fractional parts with a bubble sort (the paper's choice,
 * Sec. 4.2 footnote), walks the vertices one axis at a time (Remark 2), loads every
 * feature and adds every gradient term separately.  Same arithmetic and results as
 * sxe_encode_fwd / sxe_encode_bwd; requires kind = SXE_SIMPLEX, SXE_INDEX_HASH and
 * binary32 tables and output (else SXE_EUNSUPPORTED).  out [n_points][L*F] is overwritten; grad is a dense
 * [L][T][F] binary32 array, accumulated. */
sxe_status sxe_encode_plain_fwd(const sxe_encoder* enc, const float* x, int64_t n_points,
                                const float* tables, float* out, void* stream);
sxe_status sxe_encode_plain_bwd(const sxe_encoder* enc, const float* x, int64_t n_points,
                                const float* dout, float* grad, void* stream);

/* ------------------------------------------------------------------------ */
/* Volumetric rendering with the encodings (Sec. 6.2, Eq. 5).                 */
/* ------------------------------------------------------------------------ */

/* Ray samples: for ray r with origin o[r][3], direction d[r][3] and interval
 * [t_near[r], t_far[r]], delta[r] = (t_far - t_near) / S and sample k at
 * x[r*S + k][3] = o + t_k d, t_k = t_near + (k + 1/2) delta, each binary32 operation
 * rounded once in this order (no contraction).  The paper does not state its sampling;
 * this is the midpoint rule on S equal segments.  x [n_rays*S][3] and delta [n_rays]
 * binary32 are overwritten.  1 <= S <= 2^20. */
sxe_status sxe_vr_samples(const float* origins, const float* dirs, const float* t_near,
                          const float* t_far, int64_t n_rays, int32_t n_samples, float* x,
                          float* delta, void* stream);

/* Field head between the density and the colour network (Instant-NGP's layout, which
 * Sec. 6.2 builds on): from the density network's 16 binary32 outputs per sample,
 * density_out [n_rays*S][16] (16-byte aligned), writes sigma [n_rays*S] = exp(min(v_0, 15))
 * and the colour network's input color_in [n_rays*S][32] of `dtype` (SXE_F16 / SXE_BF16,
 * 16-byte aligned): the 16 outputs, then the 16 real spherical harmonics of degree <= 3
 * (l-major, m = -l..l; orthonormal, Condon-Shortley phase folded in) of the ray's unit
 * direction dirs [n_rays][3]. */
sxe_status sxe_vr_field(const float* density_out, const float* dirs, int64_t n_rays,
                        int32_t n_samples, int32_t dtype, float* sigma, void* color_in,
                        void* stream);

/* Front-to-back compositing of Eq. 5 for a field constant on each segment:
 *   T_k = exp(-sum_{j<k} sigma_j delta), w_k = T_k (1 - exp(-sigma_k delta)),
 *   color[r][c] = sum_k w_k sigmoid(rgb_logits[r*S+k][c]).
 * sigma [n_rays*S] >= 0, rgb_logits [n_rays*S][3], delta [n_rays] binary32.  Writes
 * color [n_rays][3]; transmittance [n_rays] = exp(-sum_k sigma_k delta) and
 * weights [n_rays*S] = w_k if not NULL.  One warp per ray (a shuffle scan of sigma delta). */
sxe_status sxe_vr_composite(const float* sigma, const float* rgb_logits, const float* delta,
                            int64_t n_rays, int32_t n_samples, float* color,
                            float* transmittance, float* weights, void* stream);

/* Backward of sxe_vr_composite for upstream colour gradients dcolor [n_rays][3]: with
 * w_k = T_k alpha_k and P_k = sum_{i<=k} w_i c_i,
 *   dsigma[k] = delta sum_c dcolor_c (T_{k+1} c_k,c - (color_c - P_k,c)),
 *   dlogits[k][c] = dcolor_c w_k c_k,c (1 - c_k,c),
 * (the derivative of Eq. 5's quadrature; the paper does not state it).  color [n_rays][3] is the
 * forward pass's output; sigma, rgb_logits, delta as in sxe_vr_composite.  Writes dsigma
 * [n_rays*S] and dlogits [n_rays*S][3] binary32.  One warp per ray. */
sxe_status sxe_vr_composite_bwd(const float* sigma, const float* rgb_logits, const float* delta,
                                const float* color, const float* dcolor, int64_t n_rays,
                                int32_t n_samples, float* dsigma, float* dlogits, void* stream);

/* Backward of sxe_vr_field: the gradient of the density network's 16 outputs,
 *   dv[p][j] = dcolor_in[p][j] (j < 16) + (j == 0 and v_0 < 15 ? dsigma[p] sigma[p] : 0)
 * from the colour network's input gradient dcolor_in [n_rays*S][32] (binary32, 16-byte aligned),
 * dsigma, sigma [n_rays*S] and the forward density outputs density_out [n_rays*S][16]; the
 * harmonics take no gradient.  dv [n_rays*S][16] binary32 (16-byte aligned), overwritten. */
sxe_status sxe_vr_field_bwd(const float* dcolor_in, const float* dsigma, const float* sigma,
                            const float* density_out, int64_t n_rays, int32_t n_samples, float* dv,
                            void* stream);

/* ------------------------------------------------------------------------ */
/* Tiny fully connected network (Sec. 5 d-e; about 7k weights, Sec. 6.1).     */
/* ------------------------------------------------------------------------ */

/* n_in inputs -> n_hidden hidden layers of `width` ReLU units -> n_out linear
 * outputs, no biases.  Supported: width = 64, n_in in {16, 32, 64},
 * 1 <= n_hidden <= 3, 1 <= n_out <= 16, dtype SXE_F16 or SXE_BF16 (tensor-core
 * operands; accumulation is binary32).
 * Weight layout (`weights`, dtype; `dweights`, binary32): the matrices
 * W_0 [width][n_in], W_1..W_{n_hidden-1} [width][width], W_out [n_out][width]
 * stored back to back, each row-major [fan_out][fan_in]. */
typedef struct {
  int32_t n_in;
  int32_t width;
  int32_t n_hidden;
  int32_t n_out;
  int32_t dtype;
} sxe_mlp_desc;

/* Number of weights of the network (host). */
int64_t sxe_mlp_n_params(const sxe_mlp_desc* desc);

/* Forward pass.
 *   in   [n_points][n_in] of desc.dtype
 *   out  [n_points][n_out] binary32
 *   act  optional [n_hidden][n_points][width] of desc.dtype receiving the
 *        post-ReLU hidden activations; NULL skips. */
sxe_status sxe_mlp_fwd(const sxe_mlp_desc* desc, const void* weights, const void* in,
                       int64_t n_points, float* out, void* act, void* stream);

/* The field between the encoding and the compositing in one kernel: the density network
 * (dd: n_in -> 64 -> 16, weights Wd), sigma = exp(min(v_0, 15)) and the colour network's
 * input [v_0..v_15, SH(d)] (as sxe_vr_field, kept in shared memory), then the colour network
 * (dc: 32 -> ... -> n_out, weights Wc, same dtype).  enc [n_rays*S][n_in] of the network
 * dtype (16-byte aligned rows), dirs [n_rays][3]; writes sigma [n_rays*S] and
 * logits [n_rays*S][dc.n_out] binary32.  Same results as sxe_mlp_fwd, sxe_vr_field and
 * sxe_mlp_fwd in sequence, bit for bit.  Volumetric rendering, Sec. 6.2. */
sxe_status sxe_vr_field_mlp(const sxe_mlp_desc* density, const void* Wd,
                            const sxe_mlp_desc* color, const void* Wc, const void* enc,
                            const float* dirs, int64_t n_rays, int32_t n_samples, float* sigma,
                            float* logits, void* stream);

/* sxe_vr_field_mlp that also writes the intermediates a training step's backward reads: the
 * density network's 16 outputs density_out [n_rays*S][16] binary32 (as sxe_mlp_fwd writes them)
 * and the colour network's input color_in [n_rays*S][32] of the network dtype (as sxe_vr_field
 * writes it), both 16-byte aligned and required when n_rays > 0.  Every output equals that of the
 * three launches bit for bit (which is what runs where the fused kernel does not apply). */
sxe_status sxe_vr_field_mlp_saved(const sxe_mlp_desc* density, const void* Wd,
                                  const sxe_mlp_desc* color, const void* Wc, const void* enc,
                                  const float* dirs, int64_t n_rays, int32_t n_samples, float* sigma,
                                  float* logits, float* density_out, void* color_in, void* stream);

/* Size in bytes of the workspace sxe_mlp_bwd needs for n_points (host). */
int64_t sxe_mlp_bwd_workspace_bytes(const sxe_mlp_desc* desc, int64_t n_points);

/* Backward pass for upstream gradient dout [n_points][n_out] (binary32).  The
 * hidden activations are recomputed on chip from `in` (no activation buffer).
 * The gradient is multiplied by `loss_scale` (a power of two keeps this exact)
 * before it is rounded to desc.dtype for the tensor cores, and every binary32
 * result is divided by it again.
 *   din        optional [n_points][n_in] binary32, overwritten with dL/din
 *   dweights   binary32, same layout as the weights, accumulated (+=)
 *   workspace  device scratch of sxe_mlp_bwd_workspace_bytes() bytes; the
 *              per-block weight-gradient partials are summed in a fixed order,
 *              so dweights is deterministic.  SXE_ENOMEM if it is too small. */
sxe_status sxe_mlp_bwd(const sxe_mlp_desc* desc, const void* weights, const void* in,
                       const float* dout, float loss_scale, int64_t n_points,
                       float* din, float* dweights, void* workspace, int64_t workspace_bytes,
                       void* stream);

/* Forward pass, L2 loss and backward pass in one sweep over the points (Sec. 6.1
 * image fitting): with y the network output, the upstream gradient is
 * dy = 2 (y - target) / (n_points*n_out); *sq_sum (one binary32 device
 * scalar) is overwritten with the batch's sum of squared residuals, summed in a
 * fixed order (n_points = 0: *sq_sum = 0, when sq_sum is not NULL, and nothing else is
 * written).  Other arguments as sxe_mlp_bwd. */
sxe_status sxe_mlp_train_l2(const sxe_mlp_desc* desc, const void* weights, const void* in,
                            const float* target, float loss_scale, int64_t n_points,
                            float* din, float* dweights, float* sq_sum,
                            void* workspace, int64_t workspace_bytes, void* stream);

/* sxe_mlp_train_l2 on one part of a batch that is processed in several calls (the points of a
 * step split so that one part's network pass can overlap another part's table backward, or the
 * shard of one rank in data-parallel training): the upstream gradient is normalised by the whole
 * batch, dy = 2 (y - target) / (batch_points * n_out), so that the parts' weight gradients,
 * accumulated into the same dweights (+=), sum to the batch's; *sq_sum is overwritten with this
 * part's sum of squared residuals.  SXE_EINVAL if n_points > batch_points; n_points = 0 sets
 * *sq_sum = 0 (when sq_sum is not NULL) and enqueues nothing else.  Other arguments as
 * sxe_mlp_train_l2.  Sec. 6.1's L2 loss over the batch. */
sxe_status sxe_mlp_train_l2_part(const sxe_mlp_desc* desc, const void* weights, const void* in,
                                 const float* target, float loss_scale, int64_t n_points,
                                 int64_t batch_points, float* din, float* dweights, float* sq_sum,
                                 void* workspace, int64_t workspace_bytes, void* stream);

/* sxe_mlp_train_l2 without a caller-provided workspace, for callers that cannot
 * allocate device memory: code running under another framework's allocator that owns
 * all device memory, real-time or embedded loops where an allocation may block or fail,
 * and code that must not allocate while a stream is being captured.  The paper has no
 * counterpart; this is an interface convenience of this library.
 * The per-CTA weight-gradient partials live in a fixed array inside the library's own
 * device memory: 2^21 binary32 values (8 MiB), held on every GPU that loads the library
 * until the process exits.  If a network needs more than that per CTA the call returns
 * SXE_ENOMEM; otherwise the persistent grid is reduced to what the array holds.
 * The first call on each device looks up the array's device address (with that device
 * current) and caches it, so make one call before any stream capture begins.
 * Every call shares the array and leaves its last contents in it; nothing in it needs to
 * start at zero.  Calls whose kernels overlap on the GPU (unordered streams) race on the
 * array: serialise them.  Results equal sxe_mlp_train_l2's up to the summation order of
 * the partials. */
sxe_status sxe_mlp_train_l2_static(const sxe_mlp_desc* desc, const void* weights, const void* in,
                                   const float* target, float loss_scale, int64_t n_points,
                                   float* din, float* dweights, float* sq_sum, void* stream);

/* sxe_mlp_train_l2 writing din grouped: column c of dL/din goes to
 * din[((c / din_group) * n_points + p) * din_group + c % din_group], i.e. [n_in/g][P][g];
 * with g = F of the encoder that is dL/d(encoding) level-major, [L][P][F].  din_group is
 * 1, 2, 4 or 8 and divides n_in; din is required.  Other arguments as sxe_mlp_train_l2. */
sxe_status sxe_mlp_train_l2_grouped(const sxe_mlp_desc* desc, const void* weights, const void* in,
                                    const float* target, float loss_scale, int64_t n_points,
                                    float* din, int32_t din_group, float* dweights, float* sq_sum,
                                    void* workspace, int64_t workspace_bytes, void* stream);

/* L2 loss of the image-fitting task (Sec. 6.1): mean over n_points*n_out of
 * (y - target)^2.  Writes dy = 2 (y - target) / (n_points*n_out) (binary32,
 * overwritten) and adds the batch's sum of squared residuals to *sq_sum
 * (one binary32 device scalar). */
sxe_status sxe_loss_l2(const float* y, const float* target, int64_t n_points, int32_t n_out,
                       float* dy, float* sq_sum, void* stream);

/* ------------------------------------------------------------------------ */
/* Adam (Kingma & Ba, Algorithm 1), binary32 master copy                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  float lr;
  float beta1;
  float beta2;
  float eps;
  int32_t skip_zero_grad;  /* 1: a parameter whose gradient is exactly 0 keeps its
                              value and moments (rule used for hash-table entries) */
} sxe_adam_desc;

/* Dense step over n parameters at 1-based step t:
 *   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   param -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
 * param, m, v, grad: [n] binary32 (grad is read, then zeroed).  param_lowp:
 * optional [n] of lowp_dtype (SXE_F16 / SXE_BF16 / SXE_F32) receiving the
 * rounded new parameters; NULL skips. */
sxe_status sxe_step(const sxe_adam_desc* desc, int64_t t, int64_t n, float* param, float* m,
                    float* v, float* grad, void* param_lowp, int32_t lowp_dtype, void* stream);

/* Table step over the entries marked in `touched` (n_entries bits), for the
 * interleaved state layout state[e] = {param[F], m[F], v[F], grad[F]} (binary32,
 * 16*F bytes per entry; its gradient is what sxe_encode_bwd writes with
 * grad = state + 3F and grad_stride = 4F).  Each marked entry takes the update
 * of sxe_step with skip_zero_grad forced on (entries never marked have gradient
 * zero and are skipped by the same rule), writes table_lowp[e*F..] in
 * lowp_dtype, zeroes its gradient and clears its bit. */
sxe_status sxe_step_touched(const sxe_adam_desc* desc, int64_t t, int64_t n_entries,
                            int32_t n_features, float* state, uint32_t* touched,
                            void* table_lowp, int32_t lowp_dtype, void* stream);

/* Step counter on the device, for training loops captured into a CUDA graph (where a host-side
 * t would be frozen at capture): sxe_adam_advance increments t (int64, device) and writes the
 * bias corrections of the new t, corrections[0] = 1/(1-beta1^t) and corrections[1] =
 * 1/(1-beta2^t) (binary32, device), formed in double-word binary32 arithmetic (about 48
 * significant bits; no FP64 instruction runs on the device) and rounded once, within one binary32
 * ulp of the exactly rounded value; one thread per beta, on `stream`.  sxe_step_dev and sxe_step_touched_dev are sxe_step and sxe_step_touched with
 * the corrections read from that device array when the kernel runs. */
sxe_status sxe_adam_advance(const sxe_adam_desc* desc, int64_t* t, float* corrections, void* stream);
sxe_status sxe_step_dev(const sxe_adam_desc* desc, const float* corrections, int64_t n, float* param,
                        float* m, float* v, float* grad, void* param_lowp, int32_t lowp_dtype,
                        void* stream);
sxe_status sxe_step_touched_dev(const sxe_adam_desc* desc, const float* corrections, int64_t n_entries,
                                int32_t F, float* state, uint32_t* touched, void* table_lowp,
                                int32_t lowp_dtype, void* stream);


/* Which kernel runs the network's training pass (sxe_mlp_bwd, sxe_mlp_train_l2*),
 * process-wide: SXE_MLP_KERNEL_MMA_SYNC (warp-level mma.sync for every product) or
 * SXE_MLP_KERNEL_TCGEN05 (tcgen05.mma with TMEM accumulators; where its shared-memory plan
 * fits, two 128-point tiles in flight per SM and the weight gradients on tcgen05 too, else one
 * tile per CTA with the weight gradients on mma.sync).  SXE_MLP_KERNEL_AUTO (the default)
 * takes SXE_MLP_KERNEL_TCGEN05_3TILE for n_out <= 8, else the two-tile tcgen05 kernel where it
 * applies, else mma.sync.  All compute the same products in the same precision (fp16/bf16
 * operands, binary32 accumulation).
 * SXE_MLP_KERNEL_TCGEN05_PIPELINED: tcgen05 with one warp issuing every product of the CTA for up
 * to four 128-point tiles in flight (each tile's epilogues run in its own warpgroup), the weight
 * gradients of all tiles accumulating in one set of TMEM accumulators.
 * SXE_MLP_KERNEL_TCGEN05_3TILE: for networks with n_out <= 16 (others fall back to
 * SXE_MLP_KERNEL_TCGEN05), up to three 128-point tiles in flight per SM, each issuing its own
 * tcgen05 products, with the output layer, the loss and the output layer's backward on warp-level
 * mma.sync inside the last hidden layer's epilogue (2 NH tensor-core round trips per tile instead
 * of 2 NH + 2).  The setting also picks sxe_mlp_fwd's kernel: the three-tile kernel's forward-only
 * form under SXE_MLP_KERNEL_AUTO and SXE_MLP_KERNEL_TCGEN05_3TILE (n_out <= 16), mma.sync
 * otherwise, and sxe_vr_field_mlp's: its tcgen05 form under the same two settings (colour
 * n_out <= 8), mma.sync otherwise.  The tcgen05 kernels are persistent, one CTA per SM that needs
 * the whole SM: where network passes run beside other streams' kernels, mma.sync shares the GPU
 * better (the serving loop below takes it for its forward passes under SXE_MLP_KERNEL_AUTO).
 * Not thread-safe: set it before launching work. */
#define SXE_MLP_KERNEL_AUTO 0
#define SXE_MLP_KERNEL_MMA_SYNC 1
#define SXE_MLP_KERNEL_TCGEN05 2
#define SXE_MLP_KERNEL_TCGEN05_PIPELINED 3
#define SXE_MLP_KERNEL_TCGEN05_3TILE 4
sxe_status sxe_mlp_set_kernel(int32_t kernel);
int32_t sxe_mlp_get_kernel(void);

/* Device-side failure word: nonzero once a bounded wait inside a kernel gave up (the
 * kernel then left its loop, freed its tensor memory and returned; its outputs are not
 * valid).  Synchronous; clears the word when `clear` is nonzero. */
sxe_status sxe_device_error(int32_t* flag, int32_t clear);

/* ---- Serving: a native continuous-batching query loop for trained fields --------------
 *
 * A server answers queries "value of the field of dimension d at these points" (the forward
 * encoding, Sec. 5 a-d, then the network's forward pass) for up to one field per dimension
 * d = 2..5.  One scheduler thread owns the GPU work:
 *   - continuous batching: queued requests of the same d are merged in arrival order, up to
 *     max_batch_points, into one batch whenever a stream slot is free;
 *   - admission by memory: a batch runs only if its device buffers (points, encoding, values)
 *     fit in the caller's arena next to the batches in flight, else it waits for completions;
 *   - overlap: each batch runs on its own stream slot (host-to-device copies of its requests'
 *     points, the two kernels, device-to-host copies of the values), and a host callback on that
 *     stream completes its requests; the network's forward pass runs on the mma.sync kernel
 *     under SXE_MLP_KERNEL_AUTO (its blocks share SMs with the other slots' kernels), on the
 *     three-tile tcgen05 kernel under SXE_MLP_KERNEL_TCGEN05_3TILE;
 *   - priority: requests of at most priority_points points are batched only with each other,
 *     up to that size, and run on the slot's high-priority stream, so the GPU's block scheduler
 *     serves them ahead of the blocks of large batches; copies go in pieces of at most 4 MB.
 * A point's value depends only on that point, so a merged request's values equal those it gets
 * alone.  The library allocates no device memory: the arena is the caller's. */
typedef struct sxe_server sxe_server;
typedef struct {
  void* arena;                /* device buffer the batches' buffers are carved from (caller-owned) */
  int64_t arena_bytes;        /* its size: the admission budget */
  int32_t n_slots;            /* batches in flight at most (one CUDA stream each), 1..16 */
  int64_t max_batch_points;   /* largest merged batch (and largest request), >= 1 */
  int64_t priority_points;    /* requests of at most this many points form their own batches,
                                 run on high-priority streams, so that small queries overtake
                                 large ones (0: one class, every batch at normal priority) */
} sxe_server_desc;

/* Creates a stopped server on the current device (streams created here). */
sxe_status sxe_server_create(const sxe_server_desc* desc, sxe_server** out);
/* Registers the field of dimension enc's d: its encoder, low-precision tables [L][T][F] (device),
 * network and weights (device).  The encoder's output type must be the network's dtype and its
 * L*F outputs the network's inputs.  Before sxe_server_start only; the handles and buffers must
 * outlive the server. */
sxe_status sxe_server_add_field(sxe_server* srv, const sxe_encoder* enc, const void* tables,
                                const sxe_mlp_desc* mlp, const void* weights);
/* Starts the scheduler thread (SXE_ENOMEM if it cannot be created); SXE_EINVAL if the server
 * is already running or has no field.  A stopped server may be started again. */
sxe_status sxe_server_start(sxe_server* srv);
/* Queues a request: n_points points x_host [n][d] binary32 and their values y_host [n][n_out]
 * binary32, both host memory (pinned for asynchronous copies) that must stay valid until the
 * request completes.  *request_id receives its id.  SXE_EINVAL (and no request) for a stopped
 * server, an unknown d, n_points < 1 or above max_batch_points, a request whose buffers could
 * never fit in the arena, or NULL buffers; SXE_ENOMEM if the host cannot hold the request.
 * Thread-safe. */
sxe_status sxe_server_submit(sxe_server* srv, int32_t d, const float* x_host, int64_t n_points,
                             float* y_host, int64_t* request_id);
/* Waits up to timeout_us microseconds (0: just polls) for a request.  *state: 0 still pending,
 * 1 done (y_host holds its values), 2 failed (sxe_last_error says why).  For states 1 and 2,
 * *latency_s (optional) receives submit-to-completion time in seconds and the id is retired.
 * Thread-safe; releases no GIL of its own (callers from Python should not hold one). */
sxe_status sxe_server_wait(sxe_server* srv, int64_t request_id, int64_t timeout_us, int32_t* state,
                           double* latency_s);
/* Stops the scheduler: with drain != 0 after every queued request has run, else queued
 * requests fail; batches in flight always complete.  Thread-safe: a second caller returns once
 * the first has stopped the server. */
sxe_status sxe_server_stop(sxe_server* srv, int32_t drain);
/* Batches launched so far and the largest arena footprint in flight. */
sxe_status sxe_server_stats(const sxe_server* srv, int64_t* n_batches, int64_t* peak_bytes);
/* Stops (draining) if running, waits for its streams and releases the server.  No other call
 * on the same server may run concurrently with it or follow it. */
sxe_status sxe_server_destroy(sxe_server* srv);

/* Diagnostic of the bounded waits: runs, on `stream`, one mbarrier wait of the kind every
 * tcgen05 kernel of the library uses (suspended polls, given up after `limit_ns` nanoseconds of
 * global time).  With expect_timeout != 0 nothing ever arrives on the barrier, so the wait gives up
 * and raises the device error word (read it with sxe_device_error); with expect_timeout == 0 the
 * barrier's phase completes first and the word is left as it is.  Either way the kernel returns
 * and the context stays usable.  limit_ns must lie in (0, 2e9]: SXE_EINVAL otherwise. */
sxe_status sxe_selftest_wait(int32_t expect_timeout, int64_t limit_ns, void* stream);

/* Thread-local message describing the last failing call on this thread ("" if none). */
const char* sxe_last_error(void);

/* Library version string. */
const char* sxe_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SIMPLEXENC_H */
