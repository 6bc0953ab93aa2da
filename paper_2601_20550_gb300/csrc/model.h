// Host-side model description shared by the C-ABI layer and the kernels' launch
// code.  Built once per model by build_model() (model.cpp).
#pragma once

#include <cstdint>
#include <vector>

#include "heom2dvs.h"

namespace heom {

struct ModeBasis {
  int n = 0;                    // kept levels
  std::vector<double> E;        // energies (rad/fs)
  std::vector<double> q[5];     // q^k, k = 1..4, n x n row-major
};

struct Model {
  int n_modes = 0, d = 0, depth = 0, precision = 0;
  double beta = 0.0;            // fs/rad
  std::vector<int> dims, stride;
  std::vector<ModeBasis> modes;
  std::vector<double> H, mu, mu_plus;          // d x d
  std::vector<std::vector<double>> Vloc;       // per mode n_s x n_s
  std::vector<double> lambda;                  // per mode reorganisation energy (rad/fs)
  // bath exponentials j: mode, nu, Re c, Im c
  int n_exp = 0;
  std::vector<int> exp_mode;
  std::vector<double> exp_nu, exp_re, exp_im;
  // hierarchy
  int n_ado = 0;
  std::vector<int32_t> ado, up, down;          // n_ado x n_exp
  std::vector<double> decay;                   // sum_j n_j nu_j
  std::vector<int32_t> nb_off, nb_idx;         // per (ado, mode) coupling lists
  std::vector<double> nb_cA, nb_cB;
  // coupling eigenbasis: v_s = U_s diag(lam_s) U_s^T per mode; U = U_0 x U_1 x ...
  std::vector<std::vector<double>> vb_lam;     // per mode, n_s eigenvalues
  std::vector<double> vb_U;                    // d x d
  std::vector<double> vb_H, vb_mu, vb_mu_plus; // U^T X U
};

// Coupling-eigenbasis quantities (fills vb_* of M).
void build_coupling_basis(Model &M);

void jacobi_eigh(std::vector<double> &A, int n, std::vector<double> &w, std::vector<double> &Z);
void pade_bose(int N, std::vector<double> &xi, std::vector<double> &eta);
Model build_model(const heom_model &m);
void build_hierarchy(Model &M);

}  // namespace heom
