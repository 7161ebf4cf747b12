/*
 * nnp.h -- C ABI of libnnp: energy and forces of an ANI-style neural-network
 * potential on one B300 GPU (sm_103a).
 *
 * What the library computes.  The machine-learning part of an ML/MM energy,
 * E_ML({r_i}, {Z_i}) (paper, Theory, Eq. 1), for the atoms handed to it, and
 * the forces F_i = -dE_ML/dr_i (Eq. 2).  Inputs are the ones the paper's
 * interface gives a model (Methods, "The nnpot Interface in GROMACS"):
 * atomic numbers, positions and the periodic box.  E_ML = sum_i E_i with
 * E_i = MLP_{s_i}(G_i): G_i is the ANI atomic environment vector (radial and
 * angular symmetry functions with cosine cutoffs) and MLP_s a per-element
 * network D -> h1 -> h2 -> h3 -> 1 with CELU activations.
 *
 * Units: Angstrom, eV, eV/Angstrom.  Unit conversion (GROMACS uses nm and
 * kJ/mol) is the caller's job.
 *
 * Threading and streams.  A context is not thread-safe; use one context per
 * host thread / CUDA stream.  All work runs on the context's stream.
 *
 * Pointers.  Arrays of positions, atomic numbers, energies and forces may be
 * host or device pointers (detected with cudaPointerGetAttributes).  Host
 * pointers are staged through pinned buffers; device pointers are read and
 * written in place.  Page-locked host positions and atomic numbers
 * (cudaHostAlloc'd or registered) given to nnp_eval or nnp_eval_batch are
 * read in place by the device during the call, outside the pair-list and
 * embedding entry points.  Boxes are always host pointers.  The caller owns
 * every pointer it passes; the library never keeps one after a call returns.
 *
 * Errors.  Every call returns an nnp_status; no exception crosses the ABI and
 * no GPU trap is used.  nnp_last_error() gives a one-line message.  Device
 * checks (unknown atomic number, non-finite position, neighbour-list
 * overflow) raise flags that the synchronous calls read back; a
 * neighbour-list overflow makes nnp_eval grow its lists and evaluate again.
 */
#ifndef NNP_H
#define NNP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nnp_ctx nnp_ctx;

typedef enum {
    NNP_OK = 0,
    NNP_ERR_INVALID_ARG = 1,     /* null pointer, n <= 0, non-finite position, bad box */
    NNP_ERR_UNKNOWN_SPECIES = 2, /* an atomic number outside the configured species */
    NNP_ERR_UNSUPPORTED = 3,     /* cell height < radial cutoff, layer sizes, a triclinic
                                    box where only orthorhombic ones are taken */
    NNP_ERR_CAPACITY = 4,        /* neighbour lists overflowed (async path) or > max */
    NNP_ERR_CUDA = 5,            /* a CUDA runtime call failed */
    NNP_ERR_TIMEOUT = 6,         /* a bounded device wait expired */
    NNP_ERR_NO_WEIGHTS = 7,      /* nnp_eval before every species had weights; FP8, from nnp_sync:
                                    an asynchronous evaluation met a species that no calibration
                                    pass had seen (the next evaluation calibrates) */
    NNP_ERR_NO_STATE = 8,        /* nnp_force_match_grad before any nnp_eval */
    NNP_ERR_BOUNDS = 9           /* bounds-checked build only (NNP_CHECKED): an index read from
                                    device data was out of range; the access was skipped and the
                                    results of the call are not valid (the message names the
                                    source line and the value) */
} nnp_status;

typedef enum {
    NNP_FP32 = 0, /* FP32 descriptors and FP32 SIMT network (reference form) */
    NNP_BF16 = 1, /* FP32 descriptors, network on tcgen05 tensor cores in BF16
                     (ensemble members side by side in one launch) */
    NNP_FP8 = 2   /* as BF16, but the three forward GEMMs in FP8 E4M3 with one static
                     scale per layer and species for activations and one per output
                     column for weights: s_W[n] = max_k |W[k][n]| / 448 at
                     nnp_set_weights; activations s_x = max|x| / 448 from an FP32
                     calibration pass over the first evaluation's input (and again
                     after new weights, or when an input has a species that no pass
                     has seen: that evaluation is then calibrated and redone).  The
                     calibration pass makes that evaluation synchronous.  The backward
                     stays BF16.  Two species or more (D >= 128). */
} nnp_precision;

#define NNP_MAX_SPECIES 8
#define NNP_MAX_SHIFTS 32
#define NNP_MAX_MEMBERS 16

/* Context flags */
#define NNP_FLAG_NO_GRAPH 0x1u      /* launch kernels directly instead of a CUDA graph */
#define NNP_FLAG_NONDETERMINISTIC_BINS 0x2u /* skip the per-cell ordering pass */
#define NNP_FLAG_STAGE_EVENTS 0x4u  /* record CUDA events between pipeline stages */
#define NNP_FLAG_CHARGES 0x10u      /* reserve a charge network (nnp_set_charge_weights) for
                                       the electrostatic embedding, nnp_eval_ee; not FP8 */
#define NNP_FLAG_AUTOTUNE 0x8u      /* pick launch shapes by timing them (cached per shape bucket;
                                       file cache: environment NNP_AUTOTUNE_CACHE) */

/*
 * Model hyper-parameters and capacities.  Fill with nnp_config_init() and
 * adjust.  The descriptor follows the ANI atomic environment vector:
 *
 *   radial, neighbour j of species s_j, shift m (n_rad shifts):
 *     G_i[s_j*n_rad + m] += 1/4 exp(-eta_r (r_ij - shf_r[m])^2) fc(r_ij; rc_r)
 *   angular, unordered neighbour pair {j,k} within rc_a, shift a, sector z:
 *     G_i[n_rad*S + p(s_j,s_k)*n_ang_r*n_ang_z + a*n_ang_z + z] +=
 *       2^(1-zeta) (1 + cos(arccos(0.95 cos theta_ijk) - shf_z[z]))^zeta
 *       * exp(-eta_a ((r_ij + r_ik)/2 - shf_a[a])^2) fc(r_ij; rc_a) fc(r_ik; rc_a)
 *   fc(r; rc) = (cos(pi r / rc) + 1) / 2 for r < rc, else 0;
 *   p(s1, s2) = row-major index of the unordered species pair (s1 <= s2).
 *
 * The kernels are specialised for n_rad = 16, n_ang_r = 4, n_ang_z = 8,
 * zeta a power of two (<= 64), hidden = {160, 128, 96}, 1 <= S <= 8
 * (S = 7, D = 1008: the H, C, N, O, S, F, Cl element set of ANI-2x); other
 * values give NNP_ERR_UNSUPPORTED.  The BF16 form takes any S (above D = 128
 * layer 1 and dE/dG are streamed in chunks); the FP8 form takes S >= 2
 * (D >= 128); nnp_eval_noalloc takes S <= 4.
 */
typedef struct {
    int32_t n_species;                        /* S */
    int32_t atomic_numbers[NNP_MAX_SPECIES];  /* species s has Z = atomic_numbers[s];
                                                 must be ascending */
    double rc_r, eta_r;
    int32_t n_rad;
    double shf_r[NNP_MAX_SHIFTS];
    double rc_a, eta_a, zeta;
    int32_t n_ang_r, n_ang_z;
    double shf_a[NNP_MAX_SHIFTS];
    double shf_z[NNP_MAX_SHIFTS];
    int32_t hidden[3];
    double celu_alpha;
    int32_t precision;        /* nnp_precision */
    int64_t max_atoms;        /* capacity hint (atoms over all systems); grows on demand */
    int32_t max_systems;      /* capacity hint for nnp_eval_batch */
    int32_t nbr_capacity;     /* radial neighbours per atom; 0 = 96; grows on overflow */
    int32_t ang_capacity;     /* angular neighbours per atom; 0 = 32; grows on overflow */
    void *stream;             /* cudaStream_t to run on; NULL = the library makes one */
    uint32_t flags;           /* NNP_FLAG_* */
    int32_t n_members;        /* ensemble size M (0 or 1 = one network; at most
                                 NNP_MAX_MEMBERS; any precision, FP8 with its own
                                 activation and weight scales per member): E_i is
                                 the mean of M networks of the same shape over the
                                 shared descriptor, as in the ANI-2x model, and
                                 the forces are minus the gradient of that mean */
} nnp_config;

/* ANI-style defaults for n_species species with the given atomic numbers
 * (ascending): radial 16 shifts 0.9 + 0.26875 m, eta_r 16, rc_r 5.2;
 * angular 4 shifts 0.9 + 0.65 a, 8 sectors (2z+1) pi/16, eta_a 8, zeta 32,
 * rc_a 3.5; hidden 160/128/96; CELU alpha 0.1; FP32; capacities 4096 atoms.
 * Returns NNP_ERR_INVALID_ARG for a null cfg, S outside 1..8 or Z not
 * ascending. */
int nnp_config_init(nnp_config *cfg, int32_t n_species, const int32_t *atomic_numbers);

/* Create a context: validates cfg, allocates device workspaces for the
 * capacity hints, creates (or adopts) the stream.  *out receives the context
 * or NULL on error. */
int nnp_create(const nnp_config *cfg, nnp_ctx **out);

/* Release every device and host resource of ctx (NULL is ignored). */
void nnp_destroy(nnp_ctx *ctx);

/* Message of the last error on ctx (or of the last failed nnp_create when
 * ctx is NULL).  The string lives until the next call on ctx. */
const char *nnp_last_error(const nnp_ctx *ctx);

/* Weights of species s (index into atomic_numbers).  W[l] is row-major
 * (fan_in x fan_out) FP32: W[0] D x h1, W[1] h1 x h2, W[2] h2 x h3,
 * W[3] h3 x 1; b[l] has fan_out entries.  Host or device pointers; the data
 * are copied (and rounded to BF16/FP8 for those precisions), the caller keeps
 * ownership.  Captured graphs stay valid (weights live in fixed buffers).
 * FP8: also resets the activation scales of every species (recalibrated at the
 * next evaluation). */
int nnp_set_weights(nnp_ctx *ctx, int32_t species, const float *const W[4],
                    const float *const b[4]);

/* Weights of species s in ensemble member m (0 <= m < n_members), laid out
 * and owned as in nnp_set_weights; nnp_set_weights is member 0.  Every member
 * of every species needs weights before the first evaluation.  The output
 * layer is stored divided by M so that the members' contributions, added
 * into the same per-atom energies and descriptor gradients, give the mean.
 * NNP_ERR_INVALID_ARG for m or s out of range or a null array. */
int nnp_set_member_weights(nnp_ctx *ctx, int32_t member, int32_t species,
                           const float *const W[4], const float *const b[4]);

/* Energy and forces of one system of n atoms.
 *   pos    n x 3 positions (Angstrom), any values (wrapped into the box);
 *   Z      n atomic numbers;
 *   box    9 doubles (3 x 3 row-major, rows = cell vectors a, b, c; host
 *          pointer); orthorhombic or triclinic (right-handed), every height
 *          of the cell across two of its vectors >= rc_r; NULL = isolated
 *          system (no periodic images);
 *   energy 1 double (eV), forces n x 3 doubles (eV/Angstrom); either may be
 *          NULL to skip it.
 * Synchronous: returns after the results are written.  After an error
 * return the contents of energy and forces are unspecified. */
int nnp_eval(nnp_ctx *ctx, int64_t n, const double *pos, const int32_t *Z,
             const double *box, double *energy, double *forces);

/* As nnp_eval, with the neighbour pairs supplied by the caller instead of the
 * library's cell search (Methods: the 2026 nnpot interface passes the MD
 * engine's own pair list to the model).
 *   pairs   n_pairs x 2 int32 atom indices (i, j), host or device: every
 *           unordered pair, or periodic self-image (i, i) with a nonzero shift,
 *           exactly once (a pair listed twice counts twice);
 *   shifts  n_pairs x 3 doubles (A), host or device, or NULL for none: the
 *           pair's displacement is r_j - r_i + shift.  With a box, a shift
 *           must be a whole periodic image (integer multiples of the edges);
 *           an isolated system (box NULL) takes no shifts.
 * Pairs whose distance is at or beyond the radial cutoff are ignored, so a
 * buffered list is fine; a pair inside it enters both atoms' neighbour lists.
 * A complete list gives the cell search's neighbour sets, hence the same
 * energy and forces up to the FP32 order of the sums (list order follows
 * the fill's atomics).  NNP_ERR_INVALID_ARG for an index out of range or a
 * shift that is not a whole image; list capacities grow as for nnp_eval. */
int nnp_eval_pairs(nnp_ctx *ctx, int64_t n, const double *pos, const int32_t *Z,
                   const double *box, int64_t n_pairs, const int32_t *pairs,
                   const double *shifts, double *energy, double *forces);

/* As nnp_eval, but pos, Z, energy and forces must be device pointers and
 * the call returns without synchronising; device-side flags (unknown species,
 * non-finite position, list overflow) are reported by the next nnp_sync(). */
int nnp_eval_async(nnp_ctx *ctx, int64_t n, const double *pos, const int32_t *Z,
                   const double *box, double *energy, double *forces);

/* Maximum number of atoms of one nnp_eval_noalloc call. */
#define NNP_NOALLOC_MAX_ATOMS 1024

/* Energy and forces of one periodic system without allocating any device
 * memory.  For callers that must not call cudaMalloc once a run is under way,
 * such as an MD engine that hands the GPU's free memory to its own pool at
 * start-up: a mid-run allocation can then fail, and it can stall the device
 * while the engine's other streams are busy.  Create the context and set its
 * weights at start-up; afterwards this call allocates nothing.
 *   Same meaning as nnp_eval for one periodic system, with n <=
 *   NNP_NOALLOC_MAX_ATOMS (larger n: NNP_ERR_CAPACITY), pos, Z, energy and
 *   forces device pointers, box a host pointer (orthorhombic, edges >= rc_r),
 *   FP32 contexts of at most 4 species only (else NNP_ERR_UNSUPPORTED;
 *   ensembles are fine).  At most 128 radial and 48
 *   angular neighbours per atom (more: NNP_ERR_CAPACITY, lists do not grow).
 *   Synchronous: it reads the device flags back and waits for the context's
 *   stream, so it cannot be called while that stream is being captured.  It
 *   runs on the context's stream and leaves the context's own buffers, graph
 *   and last-evaluation state untouched.  A box given as a device pointer is
 *   rejected (NNP_ERR_INVALID_ARG).
 * All per-call scratch lives in one fixed device array of the library (about
 * 6 MiB).  nnp_create looks up its address on the context's device, which
 * places the array in that device's memory; it then stays there until the
 * process exits.  Create the context before handing the GPU's free memory to
 * another pool.  Every call shares the array: calls that overlap on the GPU
 * (other streams, contexts or threads) race and give wrong results.
 * The paper has no counterpart of this entry point. */
int nnp_eval_noalloc(nnp_ctx *ctx, int64_t n, const double *pos, const int32_t *Z,
                     const double *box, double *energy, double *forces);

/* Wait for the context's stream and report device-side flags raised by the
 * asynchronous evaluations since the last check (they accumulate until this
 * call reads and clears them).  A list overflow grows the capacity for the
 * next evaluation and returns NNP_ERR_CAPACITY: results since the last check
 * are not valid. */
int nnp_sync(nnp_ctx *ctx);

/* B independent systems in one pass (one CUDA graph launch).
 *   offsets  B+1 host int64, offsets[0] = 0, system b owns atoms
 *            [offsets[b], offsets[b+1]) of pos/Z/forces;
 *   boxes    B x 9 host doubles (each as in nnp_eval; NULL = all isolated);
 *   energies B doubles. */
int nnp_eval_batch(nnp_ctx *ctx, int32_t B, const int64_t *offsets, const double *pos,
                   const int32_t *Z, const double *boxes, double *energies, double *forces);

/* As nnp_eval_batch, but pos, Z, energies and forces must be device pointers
 * and the call returns without synchronising (flags: see nnp_sync).  Boxes
 * are host pointers and must be given (periodic systems). */
int nnp_eval_batch_async(nnp_ctx *ctx, int32_t B, const int64_t *offsets, const double *pos,
                         const int32_t *Z, const double *boxes, double *energies, double *forces);

/* Number of network parameters: M * S * sum_l (fan_in*fan_out + fan_out) for
 * an ensemble of M members (M = 1 otherwise), packed member by member, within
 * a member species by species, each as W1 b1 W2 b2 W3 b3 W4 b4 (each W
 * row-major fan_in x fan_out). */
int64_t nnp_param_count(const nnp_ctx *ctx);

/* Weight gradient of a force loss L(F) (force matching, the training signal
 * of Eq. 2's forces): writes grad = dL/dtheta = sum_i v_i . dF_i/dtheta
 * (nnp_param_count doubles, host or device, layout as above) for the system(s)
 * of the last nnp_eval / nnp_eval_batch on ctx, whose configuration the
 * context keeps.  Pass either
 *   v    = dL/dF (n x 3, host or device) for any loss, Fref = NULL; or
 *   Fref = reference forces (n x 3): then L = |F - Fref|^2 / (3n), v =
 *          2 (F - Fref) / (3n), and *loss (if non-NULL) receives L.
 * F and the gradient are computed in the FP32 form (whatever the context's
 * precision) with FP64 sums: directional derivative of the descriptors along
 * v, then forward-over-reverse through the per-element networks.  For an
 * ensemble, F is the members' mean and member m's block of grad is the
 * gradient with respect to the weights given for member m. */
int nnp_force_match_grad(nnp_ctx *ctx, const double *v, const double *Fref, double *loss,
                         double *grad);

/* ML/MM mechanical embedding (Sec. Methods, the nnpot interface and its
 * link-atom equation).  The NNP sees the ML group plus one link atom per cut
 * ML-MM bond; the rest of the n_total-atom system is MM and gets no force
 * from here except through the links.
 *   pos, Z     n_total x 3 doubles (A) and n_total atomic numbers of the whole
 *              system (host or device);
 *   box        as in nnp_eval (3 x 3 rows; orthorhombic only; NULL = open);
 *   ml_index   n_ml distinct indices into [0, n_total) (host or device): the
 *              group, in the order the NNP sees it;
 *   link_ml, link_mm  n_link atom pairs of the cut bonds (host or device):
 *              link_ml[l] in the group, link_mm[l] outside it;
 *   link_d     n_link distances d (A) of the link atoms from their ML atoms,
 *              or NULL for 1 A each; link_Z the link atoms' atomic number
 *              (<= 0: hydrogen).
 * Link atom l sits at r_L = r_ML + d (r_MM - r_ML) / |r_MM - r_ML| (minimum
 * image of r_MM - r_ML in the box) and is evaluated as an ordinary ML atom,
 * after the group's atoms.  Outputs: *energy (eV) of the subsystem and
 * forces (n_total x 3, eV/A, host or device, overwritten): the group's atoms
 * get their own NNP force, atoms outside the group zero, and each link
 * atom's force F_L is passed on by the chain rule:
 *   F_MM += (d / |R|) (F_L - u (u . F_L)),  F_ML += F_L - (that),  u = R / |R|.
 * Errors: NNP_ERR_INVALID_ARG for an index out of range, a repeated group
 * index, a link whose ML atom is outside the group or whose MM atom is
 * inside it, d <= 0, or a zero-length bond; NNP_ERR_UNSUPPORTED for a
 * non-orthorhombic box.  Synchronous on the context's stream. */
int nnp_eval_mlmm(nnp_ctx *ctx, int64_t n_total, const double *pos, const int32_t *Z,
                  const double *box, int64_t n_ml, const int64_t *ml_index, int32_t n_link,
                  const int64_t *link_ml, const int64_t *link_mm, const double *link_d,
                  int32_t link_Z, double *energy, double *forces);

/* Charge network of species s for the electrostatic embedding (context
 * created with NNP_FLAG_CHARGES; else NNP_ERR_UNSUPPORTED): a per-element
 * network of the energy network's shape on the same descriptor whose output
 * is the atom's in vacuo charge (e).  Layout and ownership as in
 * nnp_set_weights; not averaged over an ensemble. */
int nnp_set_charge_weights(nnp_ctx *ctx, int32_t species, const float *const W[4],
                           const float *const b[4]);

/* Electrostatic embedding (Methods, the nnpot interface: the model predicts
 * in vacuo charges of the ML region, which interact with the MM point
 * charges, and the MM atoms receive forces).  Readings of what the paper
 * leaves open:
 *   q_i  = charge network of atom i's species on G_i, shifted to the total
 *          charge: q'_i = q_i - (sum_k q_k - total_charge) / n;
 *   E    = E_NNP + k_e sum_i sum_J q'_i Q_J / |r_J - r_i| over every MM charge
 *          J (k_e = 14.3996454784 eV A / e^2; with a box, the minimum image);
 *   no polarisation term.
 *   pos, Z, box, energy, forces  the ML atoms, as in nnp_eval (one system;
 *          box orthorhombic or NULL; forces include the embedding's);
 *   mm_pos n_mm x 3 doubles (A), mm_q n_mm charges (e), host or device
 *          (n_mm = 0 allowed);
 *   mm_forces n_mm x 3 doubles (eV/A), charges n doubles (q'), host or
 *          device, either may be NULL.
 * NNP_ERR_NO_WEIGHTS if a species lacks charge weights, NNP_ERR_UNSUPPORTED
 * for a triclinic box.  Synchronous on the context's stream. */
int nnp_eval_ee(nnp_ctx *ctx, int64_t n, const double *pos, const int32_t *Z, const double *box,
                int64_t n_mm, const double *mm_pos, const double *mm_q, double total_charge,
                double *energy, double *forces, double *mm_forces, double *charges);

/* Per-atom energies E_i (eV) of the last evaluation, in input order
 * (n doubles for nnp_eval, offsets[B] for nnp_eval_batch), host pointer.
 * Synchronises the context's stream. */
int nnp_atom_energies(nnp_ctx *ctx, double *out);

/* Self-tests of the library's failure handling (no GPU fault is involved).
 *   NNP_SELFTEST_WAIT_TIMEOUT: one kernel waits, with the same bounded wait as
 *   the tensor-core network's, on a barrier that nothing completes; the wait
 *   gives up after 2 ms, raises the device timeout flag and returns.  The call
 *   then returns NNP_ERR_TIMEOUT (the expected outcome), clears the flag, and
 *   the context stays usable; any other status means the bound failed. */
#define NNP_SELFTEST_WAIT_TIMEOUT 1
/*   NNP_SELFTEST_BOUNDS: one kernel checks an index that is out of range with
 *   the bounds-checked build's check.  A library built with NNP_CHECKED
 *   returns NNP_ERR_BOUNDS (the expected outcome) and clears the flag; the
 *   ordinary build, whose checks compile to nothing, returns
 *   NNP_ERR_UNSUPPORTED. */
#define NNP_SELFTEST_BOUNDS 2
int nnp_selftest(nnp_ctx *ctx, int32_t test);

/* Queries for tests and benchmarks. */
typedef enum {
    NNP_Q_LAUNCHES_PER_EVAL = 0,  /* kernels launched by one nnp_eval */
    NNP_Q_NBR_CAPACITY = 1,       /* current radial list capacity */
    NNP_Q_ANG_CAPACITY = 2,       /* current angular list capacity */
    NNP_Q_MAX_NBR = 3,            /* max radial neighbours seen in the last eval */
    NNP_Q_MAX_ANG = 4,            /* max angular neighbours seen in the last eval */
    NNP_Q_ROWS = 5,               /* padded rows of the last eval */
    NNP_Q_GRAPH_CAPTURES = 6,     /* CUDA graphs captured so far */
    NNP_Q_TUNE_NEIGHBOURS = 7,    /* blocks-per-SM cap of the neighbour kernel */
    NNP_Q_TUNE_DESCRIPTOR = 8,    /* ... of the descriptor kernel */
    NNP_Q_TUNE_BACKWARD = 9,      /* ... of the descriptor-backward kernel */
    NNP_Q_FP8_CALIBRATED = 10,    /* 1 once every species' FP8 activation scales are set */
    NNP_Q_TUNE_DESCRIPTOR_TILE = 11, /* row pairs per work item of the descriptor kernel
                                        (> 0: from the work queue; < 0: static order) */
    NNP_Q_TUNE_BACKWARD_TILE = 12,   /* rows per work item of the descriptor-backward kernel
                                        (-1: one row, static order) */
    NNP_Q_TUNE_NEIGHBOURS_QUEUE = 13, /* the neighbour kernel's form: bit 0 cells from the work
                                         queue (else static order), bit 1 each cell's groups of
                                         16 rows alternate between two warps */
    NNP_Q_CHECKED_BUILD = 14,        /* 1: the library was built with NNP_CHECKED (indices read
                                        from device data are bounds-checked) */
    NNP_Q_FP8_PASSES = 15            /* FP8: calibration passes run so far */
} nnp_query_key;

int nnp_query(nnp_ctx *ctx, int32_t key, int64_t *value);

/* Device durations (milliseconds) of the pipeline stages of the most recent
 * evaluation, for profiling: out[k] for stage k in the order cells (wrap,
 * bin, sort), neighbours, descriptor, network (forward, energy, backward),
 * descriptor backward (forces).  Needs a context created with
 * NNP_FLAG_STAGE_EVENTS (else NNP_ERR_UNSUPPORTED); waits for the stream.
 * Writes min(n_out, 5) entries. */
int nnp_profile_stages(nnp_ctx *ctx, double *out, int32_t n_out);

/* Device durations (milliseconds) of the stages of the most recent
 * nnp_force_match_grad, for profiling: out[k] for stage k in the order
 * forces (descriptor, networks, descriptor backward, FP32), tangent
 * descriptors (J_G v), network tangent and adjoint passes (all members),
 * weight-gradient reductions (all members).  Needs a context created with
 * NNP_FLAG_STAGE_EVENTS (else NNP_ERR_UNSUPPORTED) and a previous gradient
 * (else NNP_ERR_NO_STATE); waits for the stream.  Writes min(n_out, 4)
 * entries. */
int nnp_profile_force_match(nnp_ctx *ctx, double *out, int32_t n_out);

#ifdef __cplusplus
}
#endif

#endif /* NNP_H */
