// gint_handle.cuh -- the opaque gint_handle and the internal entry points between the
// libgint translation units.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "gint_internal.cuh"

struct gint_handle {
  int device = 0;
  GGeom geom{};
  // radial tables, (f, f') per knot
  double2 *tab64 = nullptr;
  float2 *tab32 = nullptr;
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
  int max_brick_orb = 0, max_brick_atoms = 0;
  double W = 0, W_exec = 0;
  // workspace
  float *D32 = nullptr;       // float32 copy of D blocks (FP32 SIMT mode)
  float *Dsplit = nullptr;    // tensor-core operand image of D (hi, lo)
  long long dsplit_elems = 0;
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
