// gint_handle.cuh -- the opaque gint_handle and the internal entry points between the
// libgint translation units.
#pragma once
#include <cuda_runtime.h>

#include <cuda_fp16.h>

#include <vector>

#include "gint_internal.cuh"

struct gint_handle {
  int device = 0;
  GGeom geom{};
  // radial tables, (f, f') per knot
  double2 *tab64 = nullptr;
  float2 *tab32 = nullptr;
  float2 *tab32i = nullptr;  // interleaved per-species copy of tab32 ([knot][radial]) for shaped species
  // float32 knot differences f_{k+1} - f_k formed in float64 (parallel to tab32 / tab32i): the
  // radial derivative of the float32 evaluators divides this difference by the knot spacing, and
  // a difference of two float32-rounded knot values would lose about two digits there
  float *dtab32 = nullptr;
  float *dtab32i = nullptr;
  long long nknots_i = 0;
  long long nknots = 0;
  // atoms
  double *pos_dev = nullptr;
  int *species_dev = nullptr;
  std::vector<double> pos_host;
  std::vector<int> species_host;
  std::vector<int> atom_norb, atom_off;  // per atom orbital count and global orbital offset
  int norb = 0;
  int max_species_norb = 0;
  // pair set (CSR by I, J sorted)
  int npairs = 0;
  long long nblock = 0;
  std::vector<int> pair_row, pair_col;
  std::vector<long long> pair_off;
  int *pair_row_dev = nullptr, *pair_col_dev = nullptr;
  long long *pair_off_dev = nullptr;
  int *pair_T_dev = nullptr;  // index of the transposed pair (J, I)
  int *pair_I_dev = nullptr;  // row atom I of each pair
  // neighbour structure
  int *n_at = nullptr, *n_ent = nullptr, *n_orb = nullptr;
  long long *b_at_off = nullptr, *b_ent_off = nullptr, *b_pair_off = nullptr;
  long long *scan_out = nullptr;
  int *s_atom = nullptr, *s_col = nullptr;
  long long *s_ent = nullptr;
  double *e_shift = nullptr;
  int *b_pair = nullptr;
  long long cap_slots = 0, cap_ent = 0, cap_pairtab = 0;
  long long nslots = 0, nent = 0, npairtab = 0;
  int max_brick_orb = 0, max_brick_atoms = 0, max_brick_ent = 0;
  // Slots and lattice images.  Normally a slot is an atom with every image of it that reaches the
  // brick (the images share one set of columns: Gamma point).  With `unfold` each (atom, image)
  // entry is a slot of its own, ordered by atom and then by the image's lattice vector, so that a
  // local-H tile of two slots belongs to one R.  `folded`: some slot of the current lists has
  // several images.
  bool unfold = false;
  bool folded = false;
  gint_handle *twin = nullptr;  // unfolded twin of a folded handle (built on first per-R use)
  // host copy of the descriptor's species and radial tables (to build the twin)
  std::vector<gint_species> d_sp;
  std::vector<gint_radial> d_rad;
  std::vector<std::vector<double>> d_tab;
  std::vector<double> d_pos0;  // positions at creation (they fixed the pair set)
  double d_skin = 0;
  double W = 0, W_exec = 0;
  // workspace
  float *D32 = nullptr;       // float32 copy of D blocks (FP32 SIMT mode)
  int *work_ctr = nullptr;    // dynamic brick counter of the persistent kernels
  int num_sms = 0;
  // tensor-core path (float16 3-term split)
  double phi_bound = 0;       // bound on |phi| used for the orbital scale
  std::vector<long long> tile_off;        // per pair: element offset of its padded D tile
  long long ntile_elems = 0;
  // D tiles in 128-byte core-matrix order: rows roundup(norb(I), 8), K = porb(J) (zero padded);
  // *_h2 hold the same tiles halved (diagonal chunk of the density pass)
  __half *Dt_hl = nullptr, *Dt_hl2 = nullptr;  // D tiles (hi, lo interleaved per 8 x 8 block), halved copy
  __half *zero_dev = nullptr;  // 512 zero bytes: source of the bulk copies for absent tiles
  long long *tile_off_dev = nullptr;
  float *scales = nullptr;    // device: [0] S_phi, [1] S_D (density), [2] S_Q (local H)
  int max_brick_porb = 0;     // largest padded (aligned) orbital count of a brick
  // local-H scratch: per brick, upper-triangle slot-pair tiles (float32), reduced per pair
  long long *hs_brick_off = nullptr;      // [nbricks + 1] element offset of each brick's tiles
  long long hs_elems = 0;
  float *hs = nullptr;
  int nupper = 0;                         // pairs with I <= J
  int *hu_pair = nullptr;                 // [nupper] pair index
  long long *hu_off = nullptr;            // [nupper + 1] CSR into hu_src
  long long *hu_src = nullptr;            // scratch element offset of each contribution
  uint4 *plan = nullptr;                  // per-brick plan records (brick metadata, prefetched by the kernel)
  long long *plan_off_dev = nullptr;      // [nbricks + 1] record offsets, 16-byte units
  long long tc_bytes = 0;                 // device bytes of the tensor-core workspace above
  // the neighbour structure these layouts were built for (host copies: brick slot offsets, slot atoms,
  // brick entry offsets); a rebuild for new positions that reproduces it refreshes the plan records only
  std::vector<long long> tc_at_off, tc_ent_off;
  std::vector<int> tc_satom;
  // local H per lattice vector (keys (I, J, R); built on first use by gint_hr_prepare)
  bool r_ready = false;
  int r_status = 0;           // GINT_OK, or why per-R output is unavailable for this geometry
  bool reduce_R = false;      // the next local-H reduction writes H(R) blocks (set around one call)
  bool reduce_fp64 = false;   // tensor-core local H: cross-brick sums in float64 (gint_set_reduction)
  int r_nkeys = 0, r_nupper = 0;
  long long r_nblock = 0, r_bytes = 0;
  std::vector<int> r_keys_host;         // [nkeys][5]: I, J, n1, n2, n3 (R = n1 a1 + n2 a2 + n3 a3)
  std::vector<long long> r_off_host;    // [nkeys + 1] element offset of each H(R) block
  int *r_kI = nullptr, *r_kJ = nullptr, *r_kT = nullptr, *r_kn = nullptr;
  long long *r_koff = nullptr;
  int *r_hu_key = nullptr;              // upper keys, each with its contributions:
  long long *r_hu_off = nullptr, *r_hu_src = nullptr;
  int *r_gk_off = nullptr;              // [npairs + 1]: keys of pair p are [gk_off[p], gk_off[p + 1])
  bool r_group_ok = false;              // every group of 8 consecutive pairs has at most 64 keys
  // velocity-gauge projector overlaps (set by gint_set_projectors)
  bool pb_ready = false;
  GTabs pb_tabs{};                      // projector radial metadata per species
  double2 *pb_tab64 = nullptr;          // projector tables, (f, f') per knot
  int pb_npairs = 0;
  long long pb_nelems = 0, pb_bytes = 0;
  std::vector<int> pb_pairs_host;       // [npairs][2]: projector atom I, orbital atom J
  std::vector<long long> pb_off_host;   // [npairs + 1] complex-element offset of each block
  int *pb_I = nullptr, *pb_J = nullptr, *pb_img_off = nullptr;
  long long *pb_off = nullptr;
  double *pb_img = nullptr;             // image positions of J per pair
  double *red = nullptr;      // reduction partials
  double *scal = nullptr;     // device scalars
  unsigned *err_word = nullptr;
  cudaStream_t own_stream = nullptr;

  GNbr nbr() const {
    GNbr n;
    n.b_at_off = b_at_off;
    n.b_norb = n_orb;
    n.s_atom = s_atom;
    n.s_col = s_col;
    n.s_ent = s_ent;
    n.e_shift = e_shift;
    n.b_pair_off = b_pair_off;
    n.b_pair = b_pair;
    n.pair_off = pair_off_dev;
    n.atom_species = species_dev;
    return n;
  }
};

// gint_nbr.cu
int gint_build_neighbours(gint_handle *h, cudaStream_t st);
// gint_capi.cu
int gint_reserve_nbr(gint_handle *h);
// gint_simt.cu
int gint_simt_rho(gint_handle *h, bool fp64, const double *D, double *rho, const double *V, double *F,
                  cudaStream_t st);
int gint_simt_vlocal(gint_handle *h, bool fp64, const double *V, double *H, cudaStream_t st);
int gint_convert_D32(gint_handle *h, const double *D, cudaStream_t st);
int gint_reduce_dot(gint_handle *h, const double *a, const double *b, long long n, double scale, double *out,
                    cudaStream_t st);
// gint_tc.cu
int gint_tc_rho(gint_handle *h, int precision, const double *D, double *rho, const double *V, double *F,
                cudaStream_t st);
int gint_tc_vlocal(gint_handle *h, int precision, const double *V, double *H, cudaStream_t st);
int gint_tc_batch(const gint_task *tasks, int n, int precision, cudaStream_t st, cudaEvent_t ev0,
                  cudaEvent_t ev1);
int gint_tc_check_capacity(const gint_handle *h);
int gint_tc_prepare(gint_handle *h);  // layouts and scratch of the tensor-core path (after neighbours)
int gint_tc_refresh(gint_handle *h);  // after a neighbour rebuild: plan records only, or gint_tc_prepare
void gint_tc_free(gint_handle *h);
// gint_hr.cu
int gint_hr_prepare(gint_handle *h);  // key tables of H(R) (GINT_EUNSUPPORTED if tiles mix R)
void gint_hr_free(gint_handle *h);
int gint_hr_bloch(gint_handle *h, const double *HR, int nk, const double *kf, double *Hk, cudaStream_t st);
// gint_pb.cu
int gint_pb_set(gint_handle *h, int nspecies, const gint_species *proj);
int gint_pb_run(gint_handle *h, const double A[3], double *out, cudaStream_t st);
void gint_pb_free(gint_handle *h);
