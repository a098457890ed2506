/*
 * mlpf.h -- C ABI of the B300 (sm_103a) MLPF full-event transformer forward.
 *
 * The library maps each event's variable-length set of PF elements (tracks and
 * calorimeter clusters, one 42-float feature vector each; Sec. 5.2) to a
 * per-element particle class (none, charged hadron, neutral hadron, photon,
 * electron, muon) and the regressed (pT, eta, sin phi, cos phi, E) of the MLPF
 * transformer (Sec. 5.3), plus FP64 per-event missing-pT and scalar-pT sums
 * (Sec. 3.3).  Many events are packed back to back and described by offsets.
 *
 * Conventions for every entry point:
 *  - Every call returns an mlpf_status and never aborts the process.  On a
 *    non-OK status, mlpf_last_error() returns a message (thread-local).
 *  - "device" pointers are CUDA device memory on the model's device (for
 *    instance torch tensors' data_ptr()); "host" pointers are CPU memory.
 *  - The caller owns every input and output buffer.  The model owns its
 *    weights and its workspace.
 *  - A model may be used from one host thread and one stream at a time.
 *    Different models are independent.
 */
#ifndef MLPF_H
#define MLPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlpf_model mlpf_model; /* opaque */

typedef enum {
    MLPF_OK = 0,
    MLPF_E_INVALID = 1,     /* bad argument (null pointer, size, precision) */
    MLPF_E_FORMAT = 2,      /* malformed weight blob (magic, version, shapes) */
    MLPF_E_CUDA = 3,        /* a CUDA runtime/driver call failed */
    MLPF_E_OOM = 4,         /* device allocation failed */
    MLPF_E_TIMEOUT = 5,     /* a bounded device-side wait ran out (see mlpf_sync) */
    MLPF_E_NONFINITE = 6,   /* non-finite values reached the outputs (see mlpf_sync) */
    MLPF_E_UNSUPPORTED = 7  /* precision/architecture combination not built */
} mlpf_status;

typedef enum {
    MLPF_FP32 = 0, /* plain path: SIMT FP32 FFMA GEMMs and attention, no TF32 */
    MLPF_BF16 = 1, /* tensor cores: attention in BF16 (Q, K, V, P and the QK^T / PV
                      products), FP16 operands in the embedding, projection, FFN and head
                      GEMMs; FP32 accumulation, softmax statistics, LayerNorm moments and
                      residual stream.  The per-stage rounding budget of the forward puts
                      the 16-bit error into the GEMM operands, not into the attention
                      products: BF16 GEMM operands cost the 99.9 % argmax bound.
                      The d=64, 4 x 16, FFN 256 arch-0 model runs fused persistent kernels;
                      every other model (any width with heads of 16, 32 or 64, both
                      architectures) runs the generic-width path: one tcgen05 GEMM per
                      linear layer with two-term FP16 weights (FP16 rounding plus the
                      rounding of the remainder), warp-level MMA attention */
    MLPF_FP8 = 2,  /* E4M3 GEMMs with per-tensor scales, FP16 attention (needs mlpf_calibrate_fp8);
                      the d=64, 4 x 16, FFN 256 arch-0 model only */
    MLPF_FP16 = 3  /* FP16 everywhere on the tensor-core path (attention included) */
} mlpf_precision;

/* Model configuration, as stored in the weight blob header. */
typedef struct {
    int32_t in_dim; /* 42 input features per element */
    int32_t d;      /* model width */
    int32_t heads;  /* attention heads; head width d/heads */
    int32_t ffn;    /* FFN hidden width */
    int32_t l_pid;  /* encoder blocks in the classification (PID) stack */
    int32_t l_reg;  /* encoder blocks in the regression stack */
    int32_t n_cls;  /* 6 classes: none, ch. hadron, n. hadron, photon, electron, muon */
    int32_t n_reg;  /* 5 regression outputs: pT, eta, sin phi, cos phi, E */
    int32_t act;    /* 0 = GELU (exact erf form), 1 = ReLU */
    int32_t arch;   /* 0 = one shared embedding, the regression stack reads
                       concat(x, h_pid), one 6-class head (argmax);
                       1 = the architecture as Sec. 5.3 prints it: track and cluster
                       embeddings, two parallel stacks on the same embedding, a
                       binary head (logit column 0; a particle where it is > 0, i.e.
                       score > 0.5) and a 5-class PID head (columns 1-5; class =
                       1 + argmax).  arch 1 runs on MLPF_FP32 only. */
} mlpf_config;

/*
 * Load a weight blob and create a model on CUDA device `device`.
 *
 * The blob plays the role of the paper's frozen inference graph (Sec. 8):
 *   char magic[4] = "MLPF"; int32 version = 1;
 *   int32 in_dim, d, heads, ffn, l_pid, l_reg, n_cls, n_reg, act, n_tensors;
 *   n_tensors x { char name[48]; int32 ndim; int32 shape[2]; float data[] }
 * (little endian; tensors as written by synth.pack_blob, matrices [out, in]).
 * blob: host memory, read during the call only.  *out receives the model.
 * Errors: MLPF_E_INVALID (null, nbytes too small, bad device),
 *         MLPF_E_FORMAT (magic, version, missing/extra/mis-shaped tensor,
 *         truncated data), MLPF_E_CUDA / MLPF_E_OOM.
 */
mlpf_status mlpf_load_weights(const void* blob, size_t nbytes, int device, mlpf_model** out);

/* Release a model, its weights, workspace and cached graphs.  NULL is a no-op. */
void mlpf_free(mlpf_model* m);

/* Copy the model configuration into *cfg (host). */
mlpf_status mlpf_get_config(const mlpf_model* m, mlpf_config* cfg);

/*
 * Batched forward over packed events (Sec. 5.3; inference decoding as in
 * Sec. 5.3; missing-pT sums as in Sec. 3.3).  Asynchronous on `stream`.
 *
 * x          device, [total, 42] float32 row-major, 8-byte aligned (every
 *            cudaMalloc'd or torch buffer is); event e occupies rows
 *            cu_seqlens[e] .. cu_seqlens[e+1]-1.  Feature layout: x[:,0:8]
 *            type one-hot, x[:,8] log pT, x[:,9] log E, x[:,10] eta,
 *            x[:,11:13] sin/cos phi, x[:,13:42] other features.
 * cu_seqlens device, [n_events+1] int32, cu[0] = 0, non-decreasing,
 *            cu[n_events] = total.  Empty events (N = 0) are allowed.
 * n_events, total   host scalars matching cu_seqlens.
 * max_n      host scalar >= max_e N_e (sizes launch grids), <= 65536.
 * logits     device out, [total, 6] float32 raw class scores.
 * reg        device out, [total, 5] float32 decoded (pT GeV, eta, sin phi,
 *            cos phi, E GeV) with pT = exp(x[:,8] + pT'), E = exp(x[:,9] + E').
 * cls        device out or NULL, [total] int32 argmax class, lowest index on ties.
 * event_sums device out or NULL, [n_events, 3] float64 (METx, METy, sum pT)
 *            over elements with cls != 0; phi from (sin, cos) / |(sin, cos)|.
 * stream     cudaStream_t (NULL = legacy default stream).
 *
 * total = 0 is a no-op.  Inputs are not validated on the device: offsets
 * that break the contract give undefined results (but stay in bounds of
 * the workspace sized from total/max_n/n_events).
 * Errors: MLPF_E_INVALID (null pointers, x not 8-byte aligned, negative
 *         sizes, max_n > 65536, unknown precision), MLPF_E_UNSUPPORTED (MLPF_FP8 on a model
 *         other than the d=64 one, or a 16-bit precision on a device other than sm_103),
 *         MLPF_E_OOM (workspace growth), MLPF_E_CUDA.
 * Device-side timeouts and non-finite outputs are reported by mlpf_sync().
 */
mlpf_status mlpf_forward(mlpf_model* m, int32_t precision,
                         const float* x, const int32_t* cu_seqlens,
                         int32_t n_events, int32_t total, int32_t max_n,
                         float* logits, float* reg, int32_t* cls,
                         double* event_sums, void* stream);

/*
 * Same as mlpf_forward with HOST buffers: copies x and cu_seqlens to the
 * device workspace, runs the forward and copies the outputs back; returns when
 * the host outputs are written.  Large batches are processed in chunks of
 * consecutive events (MLPF_OPT_HOST_CHUNKS) whose host-to-device copies,
 * forwards and device-to-host copies are pipelined on the caller's stream,
 * two copy streams of the model and (MLPF_OPT_HOST_STREAMS) a second compute
 * stream; the results are those of a single-chunk call
 * (an event's outputs do not depend on the other events).  x, cu_seqlens: host inputs (pinned memory lets the copies run
 * asynchronously); logits, reg: host outputs; cls, event_sums: host outputs or
 * NULL.  Errors as mlpf_forward plus those of mlpf_sync.
 */
mlpf_status mlpf_forward_host(mlpf_model* m, int32_t precision,
                              const float* x, const int32_t* cu_seqlens,
                              int32_t n_events, int32_t total, int32_t max_n,
                              float* logits, float* reg, int32_t* cls,
                              double* event_sums, void* stream);

/*
 * mlpf_forward with no device allocation: for callers that may not allocate GPU
 * memory while they run (an event loop under a caching allocator or a fixed
 * memory budget, or code that cannot afford the synchronisation a cudaMalloc
 * implies).  The paper has no counterpart; this is a library-usage variant.
 *
 * Same arguments, layouts and result as mlpf_forward for precision MLPF_BF16 or
 * MLPF_FP16 (others: MLPF_E_UNSUPPORTED).  The forward's scratch lives in one
 * file-scope device array of about 18.4 MB (held on every GPU that loads the
 * library until the process exits) instead of the model's workspace, so each
 * call takes at most 16384 elements and 64 events (larger: MLPF_E_INVALID with
 * a message).  No CUDA graph is used and nothing is allocated: not the
 * workspace, not profiling events.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) and encodes its tensor maps.  Under CUDA's lazy module
 * loading (the default) that first call may also load the library's module on
 * the device and so reserve the array there: it is the one call that can take
 * device memory, so make it before any memory-budgeted loop and before any
 * stream capture.  Later calls allocate nothing and leave the model unchanged.  Every call on a device shares the one array and
 * overwrites it: calls that overlap on the GPU (several streams, models or host
 * threads at once) race; serialise them.  Asynchronous on `stream`; device-side
 * status via mlpf_sync.
 */
mlpf_status mlpf_forward_noalloc(mlpf_model* m, int32_t precision,
                                 const float* x, const int32_t* cu_seqlens,
                                 int32_t n_events, int32_t total, int32_t max_n,
                                 float* logits, float* reg, int32_t* cls,
                                 double* event_sums, void* stream);

/*
 * Static FP8 calibration (per-tensor scales of the E4M3 GEMMs).  Runs the FP16
 * tensor-core forward on the given calibration events (device buffers, as in
 * mlpf_forward) while recording, for every GEMM input (activation), the largest
 * |value| over valid elements; sets that input's scale to amax / 448 (the
 * largest finite E4M3).  Weight scales are set at load time the same way from
 * each weight matrix.  Synchronous; must precede the first MLPF_FP8 forward
 * (otherwise MLPF_E_INVALID) and replaces earlier scales.
 */
mlpf_status mlpf_calibrate_fp8(mlpf_model* m, const float* x, const int32_t* cu_seqlens,
                               int32_t n_events, int32_t total, int32_t max_n, void* stream);

/*
 * Autotuner (no counterpart in the paper): times every attention variant (heads
 * per warpgroup x K/V pipeline depth) of `precision` on the given batch (device
 * buffers, laid out as in mlpf_forward; outputs go to the model's scratch) and
 * keeps the fastest for this model.  Models on the generic-width path: times their two
 * attention kernels instead and keeps the faster in MLPF_OPT_WIDE_ATTN_KERNEL (cache
 * key suffix "_wide").  cache_path (host string, or NULL for no
 * cache): a text file of "key variant ms" lines keyed by GPU arch, SM count, model
 * width, precision and element count rounded up to a power of two; a cached key is
 * applied without timing, a new one is appended.  Synchronous on `stream`.
 * MLPF_FP32 has nothing to tune and returns MLPF_OK.  Errors as mlpf_forward.
 */
mlpf_status mlpf_autotune(mlpf_model* m, int32_t precision, const float* x, const int32_t* cu_seqlens,
                          int32_t n_events, int32_t total, int32_t max_n, const char* cache_path,
                          void* stream);

/*
 * Anti-kt jets of every event's reconstructed particles (Sec. 3.3 and Sec. 6.2: jets
 * are clustered from the (ML)PF candidates with the anti-kt algorithm, R = 0.4 or
 * 0.8; no pileup weights).  Particles: the elements with cls != 0, pT > 0 and
 * (sin phi, cos phi) != 0, massless (px = pT c / r, py = pT s / r with r = |(s, c)|,
 * pz = pT sinh(eta), E = pT cosh(eta); the regressed E is not used).  Distances
 * d_ij = min(pT_i^-2, pT_j^-2) dR_ij^2 / R^2 (rapidity and azimuth) and d_iB =
 * pT_i^-2; E-scheme recombination (Cacciari, Salam, Soyez, JHEP 04 (2008) 063).
 * FP32 on the GPU, one CTA per event, O(N^2) per event.  Equal distances: the beam
 * distance wins, then the lower entry, entries numbered in the order the kernel keeps
 * them (by rapidity for events of at most 12,288 elements, else input order).
 * reg        device, [total, 5] decoded outputs of mlpf_forward (pT, eta, sin phi,
 *            cos phi, E); cls: device, [total] int32 classes; cu_seqlens: device,
 *            [n_events + 1] (as mlpf_forward).
 * R          distance parameter, 0 < R <= 2.
 * jets       device out, [total, 4] float32: event e's jets (px, py, pz, E) in rows
 *            cu[e] .. cu[e] + n_jets[e] - 1, in the order they leave the list.
 * n_jets     device out, [n_events] int32.
 * jet_of     device out or NULL, [total] int32: the element's jet index within its
 *            event, -1 for elements that are not particles (and for particles whose
 *            inputs are not finite enough to give a distance, which join no jet).
 * The events' CTAs run largest event first (a one-CTA sort of the element counts, for
 * up to 4,096 events; more keep the input order), so that the largest events do not
 * end the launch.  Uses a scratch of 53 bytes per element and 4 per event owned by
 * the model (grown on demand, not during graph capture).  Asynchronous on `stream`.
 * Errors: MLPF_E_INVALID (NULL
 * pointers, negative sizes, R out of range), MLPF_E_OOM, MLPF_E_CUDA.
 */
mlpf_status mlpf_cluster_jets(mlpf_model* m, const float* reg, const int32_t* cls,
                              const int32_t* cu_seqlens, int32_t n_events, int32_t total, float R,
                              float* jets, int32_t* n_jets, int32_t* jet_of, void* stream);

/*
 * Measured unit rates of `device` (no counterpart in the paper; the roofline
 * denominators of the attention kernel): results per second of the MUFU base-2
 * exponential (ex2.approx.f32) and of FP32 FMA, each from a kernel of independent
 * chains on every SM (best of three timed runs, about 1 ms each).  Either output
 * pointer (host) may be NULL.  Allocates and frees its own scratch; synchronous.
 */
mlpf_status mlpf_measure_unit_rates(int32_t device, double* ex2_per_s, double* ffma_per_s);

/*
 * The packed BF16 exponential rate of device `device` (ex2.approx.ftz.bf16x2, two
 * results per instruction), measured the same way: *results_per_s (host) receives
 * exponentials per second.  The denominator of the attention roofline for kernels
 * whose softmax numerators use packed 16-bit exponentials (the tensor-memory
 * attention kernel in BF16 and FP16).  Synchronous; allocates a small scratch.
 * Errors: MLPF_E_INVALID (NULL output), MLPF_E_CUDA, MLPF_E_OOM.
 */
mlpf_status mlpf_measure_ex2_packed_rate(int32_t device, double* results_per_s);

/*
 * Names (cap x 32 bytes, or NULL) and activation scales (cap floats, or NULL)
 * of the FP8 calibration; returns the number of activation slots, 0 before
 * calibration, -1 on error.
 */
int32_t mlpf_get_fp8_scales(const mlpf_model* m, int32_t cap, char* names, float* scales);

/*
 * Student inference with per-event fallback to the full model.  `student` runs
 * on every event (precision student_precision); an event whose mean (or, with
 * MLPF_OPT_GATE_CONFIDENCE = 1 on the student, minimum), over its elements, of
 * the student's largest class probability (max softmax of the logits) is below
 * `threshold` is rerun by `teacher` (teacher_precision) and its rows of
 * logits/reg are replaced.  Both models must use the same class-score layout
 * (arch).  Arguments as mlpf_forward, plus:
 * used_teacher  device out or NULL, [n_events] int32, 1 where the teacher ran;
 * n_fallback    host out or NULL, number of such events.
 * Synchronises `stream` once (to size the teacher's batch).  Both models must
 * live on the same device.  The paper runs the full model only; this is the
 * distilled-student extension.
 */
mlpf_status mlpf_forward_gated(mlpf_model* student, mlpf_model* teacher, float threshold,
                               int32_t student_precision, int32_t teacher_precision,
                               const float* x, const int32_t* cu_seqlens,
                               int32_t n_events, int32_t total, int32_t max_n,
                               float* logits, float* reg, int32_t* cls, double* event_sums,
                               int32_t* used_teacher, int32_t* n_fallback, void* stream);

/*
 * Training of a model with hand-written FP32 forward and backward kernels and the
 * LAMB optimizer: distillation of a (student) arch-0 model on per-element outputs
 * of a full model (mlpf_trainer_step), or supervised training of an arch-1 model
 * on per-element targets (mlpf_trainer_step_supervised).
 *
 * Loss, averaged over the batch's elements: KL(p_teacher || p_student) of the
 * class probabilities plus the sum of squared differences of the 5 raw
 * regression outputs (pT', eta, sin phi, cos phi, E'), the teacher's raw values
 * recovered from its decoded ones (pT' = log(pT / pT_elem), E' likewise; Eq. 2).
 */
typedef struct mlpf_trainer mlpf_trainer;

/* Create a trainer from a weight blob (initial weights); blob read during the call. */
mlpf_status mlpf_trainer_create(const void* blob, size_t nbytes, int device, mlpf_trainer** out);
void mlpf_trainer_free(mlpf_trainer* t);
/* Number of trainable parameters (the gradient vector's length), -1 on NULL. */
int64_t mlpf_trainer_num_params(const mlpf_trainer* t);

/*
 * One step on a packed batch (device buffers as in mlpf_forward).
 * t_logits, t_reg: device, the teacher's mlpf_forward outputs for this batch.
 * lr: learning rate of this step.  update: 0 = loss and gradients only.
 * grads_out: device or NULL, [num_params] float, the gradient in blob tensor order.
 * loss_out: host or NULL (then the call is asynchronous), the batch loss.
 */
mlpf_status mlpf_trainer_step(mlpf_trainer* t, const float* x, const int32_t* cu_seqlens,
                              int32_t n_events, int32_t total, int32_t max_n,
                              const float* t_logits, const float* t_reg, float lr,
                              int32_t update, float* grads_out, double* loss_out, void* stream);

/*
 * One supervised training step of a model of the printed architecture (arch 1:
 * binary + PID heads) on the loss of Eq. 1, averaged over the batch's elements:
 *   beta BCE(b, sigmoid(z)) + b [ -(1 - p_t)^focal_gamma log p_t
 *                                 + sqrt(pT_t) (dpT'^2 + dE'^2)
 *                                 + delta (deta^2 + dsin^2 + dcos^2) ]
 * with b = [cls_target > 0], p_t the PID softmax probability of class cls_target
 * (1..5), pT' and E' targets log(target / element value) (Eq. 2).  The paper sets
 * beta = 0.01 and weights the pT and E terms by sqrt(pT target); focal_gamma and
 * delta are unstated (2 and 1 are the readings used by the oracle).
 * cls_target: device [total] int32 in 0..5; reg_target: device [total, 5] fp32
 * (pT, eta, sin phi, cos phi, E) of the target particle (read where cls > 0).
 * Other arguments and the update as mlpf_trainer_step.  MLPF_E_UNSUPPORTED for an
 * arch-0 model.
 */
mlpf_status mlpf_trainer_step_supervised(mlpf_trainer* t, const float* x, const int32_t* cu_seqlens,
                                         int32_t n_events, int32_t total, int32_t max_n,
                                         const int32_t* cls_target, const float* reg_target, float beta,
                                         float focal_gamma, float delta, float lr, int32_t update,
                                         float* grads_out, double* loss_out, void* stream);

/*
 * Arithmetic of the trainer's products (Sec. 5.3 trains the model in mixed
 * precision).  MLPF_FP32 (default): SIMT FP32 FMAs everywhere.  MLPF_BF16 / MLPF_FP16:
 * the operands of every linear-layer GEMM (forward, input and weight gradients) are
 * rounded to that 16-bit format and multiplied on the tcgen05 tensor cores (mlpf_gemm_tc),
 * and the attention forward and backward run on warp-level tensor-core MMAs with 16-bit
 * Q, K, V, probabilities, output and score gradients; FP32 accumulation, softmax
 * statistics and log-sum-exp.  Master weights, optimizer state, activations, LayerNorm
 * and the loss stay FP32.  Takes effect from the next
 * forward or step (a pending mlpf_trainer_forward is invalidated).  A bounded wait
 * that runs out inside a tensor-core GEMM is reported as MLPF_E_TIMEOUT by the next
 * synchronous step (loss_out given).  Errors: MLPF_E_INVALID (NULL),
 * MLPF_E_UNSUPPORTED (another precision), MLPF_E_OOM (operand scratch).
 */
mlpf_status mlpf_trainer_set_precision(mlpf_trainer* t, int32_t precision);

/* Current weights as a blob (host buffer of cap bytes, or NULL to query *nbytes). */
mlpf_status mlpf_trainer_export(const mlpf_trainer* t, void* blob, size_t cap, size_t* nbytes);

/*
 * The trainer's forward and backward as separate calls, for frameworks that own
 * the loss and the optimizer (torch.autograd.Function; the paper trains with
 * LAMB, Sec. 5.3, which mlpf_trainer_step runs itself).
 *
 * mlpf_trainer_forward: the hand-written FP32 forward of the trainer's model on a
 * packed batch (device buffers as in mlpf_forward, at least one event and one
 * element), keeping every activation the backward needs in the trainer.
 *   logits  device out, [total, 6] float32 class scores;
 *   raw     device out, [total, 5] float32 raw head outputs (pT', eta, sin phi,
 *           cos phi, E'; decoded pT = exp(x[:,8] + pT'), E = exp(x[:,9] + E')).
 * mlpf_trainer_backward: the gradient of a scalar loss with respect to every
 * parameter, from dL/dlogits and dL/draw (device, [total, 6] and [total, 5]
 * float32), through the hand-written backward kernels (GEMM, LayerNorm, GELU, and
 * varlen attention recomputing the probabilities from Q, K and the saved row
 * log-sum-exp).  It must follow mlpf_trainer_forward on the same batch (the same
 * x and cu_seqlens pointers and sizes) with no other forward or step in between,
 * else MLPF_E_INVALID.  grads_out: device out, [num_params] float32 in blob tensor
 * order (overwritten).
 * mlpf_trainer_params: device copies of the flat parameter vector ([num_params]
 * float32, blob tensor order): `get` (or NULL) receives the current parameters,
 * then `set` (or NULL) replaces them.
 * All three are asynchronous on `stream`.
 */
mlpf_status mlpf_trainer_forward(mlpf_trainer* t, const float* x, const int32_t* cu_seqlens,
                                 int32_t n_events, int32_t total, int32_t max_n,
                                 float* logits, float* raw, void* stream);
mlpf_status mlpf_trainer_backward(mlpf_trainer* t, const float* x, const int32_t* cu_seqlens,
                                  int32_t n_events, int32_t total, int32_t max_n,
                                  const float* dlogits, const float* draw, float* grads_out,
                                  void* stream);
mlpf_status mlpf_trainer_params(mlpf_trainer* t, float* get, const float* set, void* stream);

/*
 * The trainer's tensor-core GEMM (the dense map of every linear layer, Sec. 5.3):
 *   C[M, N] (op)= act(A[M, K] B[N, K]^T + bias) + R
 * precision: MLPF_BF16 or MLPF_FP16 (the format of A and B), FP32 accumulation.
 * A: device [M, lda], B: device [N, ldb], 16-bit row-major, 16-byte aligned, lda and
 *    ldb multiples of 8 and >= K; K > 0 a multiple of 64 (zero-pad shorter rows).
 * C: device [M, ldc] float32 (ldc >= N).  bias: device [N] or NULL.  R: device
 *    [M, ldr] float32 or NULL.  act: -1 none, 0 GELU (erf form), 1 ReLU, applied to
 *    the product plus bias; R is added after it.
 * mode: 0 C = result, 1 C += result, 2 C += result with the K range split in chunks of
 *    kchunk (a multiple of 64; 0 = one chunk) whose partial products are added
 *    atomically (bias and R once).
 * status: device uint32 word; the value 2 is ORed into it if a bounded wait inside
 *    the kernel ran out (C is then incomplete).  Asynchronous on `stream`.
 * Errors: MLPF_E_UNSUPPORTED (precision), MLPF_E_INVALID (NULL, sizes, alignment),
 *         MLPF_E_CUDA (launch or tensor-map encoding failed).
 */
mlpf_status mlpf_gemm_tc(int32_t precision, const void* A, int64_t lda, const void* B, int64_t ldb,
                         int32_t M, int32_t N, int32_t K, float* C, int64_t ldc, const float* bias,
                         const float* R, int64_t ldr, int32_t act, int32_t mode, int32_t kchunk,
                         uint32_t* status, void* stream);

/*
 * Wait for the model's work on `stream` and report device-side status:
 * MLPF_E_TIMEOUT if a bounded wait inside a kernel ran out since the last
 * mlpf_sync (the kernel returned early; outputs are invalid), otherwise
 * MLPF_OK.  Clears the device status word.
 */
mlpf_status mlpf_sync(mlpf_model* m, void* stream);

/* Options (mlpf_set_option). */
enum {
    MLPF_OPT_USE_GRAPHS = 1,        /* 1 (default): replay CUDA graphs for repeated calls */
    MLPF_OPT_WAIT_LIMIT_NS = 2,     /* bound of every device-side wait (default 2e9 ns) */
    MLPF_OPT_DEBUG_STALL = 3,       /* 1: attention consumers wait on a barrier nothing
                                       arms, to exercise the timeout path (tests only) */
    MLPF_OPT_ATTN_CTAS_PER_SM = 4,  /* attention persistent grid size factor (autotuned) */
    MLPF_OPT_ATTN_KV_STAGES = 5,    /* read-only: K/V pipeline depth of the BF16 variant */
    MLPF_OPT_PROFILE = 6,           /* 1: CUDA events around every kernel launch (also
                                       inside captured graphs); see mlpf_profile_get */
    MLPF_OPT_ATTN_VARIANT_BF16 = 7, /* attention kernel variant of a precision,
                                       0..MLPF_ATTN_VARIANTS-1 (set by mlpf_autotune):
                                       tcgen05 with S and P in tensor memory (P the
                                       tensor-memory operand of the PV product), one
                                       warpgroup per head, an MMA warp:
                                         0 = 4 K/V stages, 1 = 6, 2 = 8;
                                       warp-level MMAs, each warp 32 rows of one head:
                                         3 = 4 stages, 4 = 8 stages (default);
                                       the same on 64-row half items, two CTAs per SM,
                                       4 stages: 5;
                                       warp-level PV with QK^T on tcgen05 (S in two
                                       tensor-memory buffers per head, read in the
                                       warp-level accumulator layout):
                                         6 = 4 stages, 7 = 8 stages;
                                       warp-level QK^T with P written to tensor
                                       memory and PV plus row sums on tcgen05 (O and
                                       l in tensor memory), an MMA warp:
                                         8 = 4 stages, 9 = 8 stages */
    MLPF_OPT_ATTN_VARIANT_FP16 = 8,
    MLPF_OPT_ATTN_VARIANT_FP8 = 9,
    MLPF_OPT_ATTN_WINDOW = 10,      /* 0 (default): full attention within each event.
                                       w > 0 (not the paper's model; an option of Sec. 9's
                                       block/sparse attention): each event's elements are
                                       ordered by eta (x[:, 10], ties by position), and
                                       query block b of 128 elements attends to key blocks
                                       b - w .. b + w only; outputs are returned in the
                                       input order.  Runs on MLPF_FP32 and on every
                                       tensor-core attention variant.  Events of at
                                       most 16384 elements (else MLPF_E_UNSUPPORTED);
                                       not available in mlpf_forward_noalloc. */
    MLPF_OPT_GATE_CONFIDENCE = 11,  /* student models in mlpf_forward_gated: event
                                       confidence = mean (0, default) or minimum (1) over
                                       the event's elements of the max softmax */
    MLPF_OPT_HOST_CHUNKS = 12,      /* mlpf_forward_host: the batch is split into this many
                                       chunks of consecutive events (element counts in the
                                       ratio 1/2 : 1 : ... : 1 : 1/2; 1..16, default 8); chunk c's input copy,
                                       forward and output copy run on three streams, so
                                       copies overlap the neighbouring chunks' compute.
                                       Batches under 65536 elements run as one chunk. */
    MLPF_OPT_HOST_STREAMS = 13,     /* mlpf_forward_host: compute streams the chunks
                                       alternate over, 1 or 2 (default 2).  With 2, odd
                                       chunks run on a second stream of the model with a
                                       second workspace (sized for the largest chunk), so
                                       a chunk's last attention items overlap the next
                                       chunk's kernels.  The results do not depend on it. */
    MLPF_OPT_WIDE_ATTN_KERNEL = 14  /* models outside the fused d = 64 kernels (generic-width
                                       tensor-core path): 0 (default) = the warp-level
                                       attention kernel (every product on warp-level MMAs);
                                       1 = the kernel with the PV products and row sums on
                                       tcgen05 for heads of 16 or 32 in groups of four heads
                                       (the warp-level kernel otherwise; slower on the
                                       models measured).  Results differ only in rounding
                                       (both are oracle-checked). */
};
#define MLPF_ATTN_VARIANTS 10
mlpf_status mlpf_set_option(mlpf_model* m, int32_t option, int64_t value);
mlpf_status mlpf_get_option(const mlpf_model* m, int32_t option, int64_t* value);

/*
 * Number of kernels launched by the most recent forward call (all precisions),
 * counted on the host at launch (a graph replay counts its kernel nodes).
 */
int64_t mlpf_last_launch_count(const mlpf_model* m);

/*
 * Per-kernel device times of the most recent forward made with MLPF_OPT_PROFILE
 * on (for a graph replay: of that replay).  Waits for the last kernel.
 * names: host out or NULL, cap x 32 bytes (NUL-terminated kernel names);
 * ms: host out or NULL, cap floats (milliseconds, CUDA-event resolution).
 * Returns the number of profiled launches (may exceed cap), 0 when profiling
 * is off, -1 on error.
 */
int32_t mlpf_profile_get(mlpf_model* m, int32_t cap, char* names, float* ms);

/* Thread-local message describing the last non-OK status of this thread. */
const char* mlpf_last_error(void);

/*
 * Evaluate an activation as a path computes it, on device arrays (a check of the
 * kernels' arithmetic; no counterpart in the paper): impl 0 = the FP32 path
 * (GELU from CUDA erff), impl 1 = the tensor-core epilogues (GELU from the
 * Abramowitz & Stegun 7.1.26 erf with MUFU reciprocal and exponential);
 * act 0 = GELU, 1 = ReLU.  y[i] = act(x[i]) for i < n, asynchronous on `stream`.
 */
mlpf_status mlpf_eval_activation(int32_t impl, int32_t act, const float* x, float* y, int32_t n,
                                 void* stream);

/*
 * Cost-balanced split of one packed batch over n_shards devices (host only, no
 * CUDA call).  Events are independent, so a batch shards with no exchange step;
 * the attention cost of an event grows as N_e^2, so each event goes, longest
 * first (largest N_e^2; equal costs in index order), to the shard whose summed
 * N^2 is smallest so far (lowest shard index on ties): the LPT rule, whose
 * largest shard is within 4/3 of the best possible split.
 * sizes: host, [n_events] element counts (>= 0); shard_of_event: host out,
 * [n_events] shard index in 0..n_shards-1; shard_cost: host out or NULL,
 * [n_shards] sum of N_e^2 of each shard.  Deterministic.
 * Errors: MLPF_E_INVALID (n_shards < 1, NULL pointers, negative sizes).
 */
mlpf_status mlpf_shard_events(const int32_t* sizes, int32_t n_events, int32_t n_shards,
                              int32_t* shard_of_event, double* shard_cost);

/* ABI version of this library (major * 100 + minor). */
int32_t mlpf_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MLPF_H */
