// Device state of the slot solver (krylov.cu) and the tensor-core Gram-Schmidt (gs_tc.cu).
#pragma once
#include <cuda_runtime.h>

namespace hh {

struct KState {
  int nrhs, t, D, maxit, maxV, maxZ, GX, GQ, scheme, passes;  // nrhs = number of slots
  double eta;
  double* tolv;            // per slot tolerance
  double2** Zcur;          // per slot: this iteration's Z block (t columns)
  double2** Vcur;          // per slot: this iteration's block of new basis vectors
  int* adm;                // per slot: 1 = being admitted now (start kernels)
  int* fin;                // per slot: 1 = being finalised now (solution kernels)
  double2** xout;          // per slot: where its solution goes
  double2* bdev;           // per slot right-hand side (slots x D)
  double* beta;
  int *done, *status, *nV, *nZ, *iters, *nacc, *amap;
  double *rho, *nu, *cs, *hist, *npart;
  double* azpart;          // per slot, new column j, CTA c of gs_wprep_kernel: its part of ||A z_j||^2
  double2 **Vptr, **Zptr;
  double2 *Hacc, *Hthis, *Hpart, *Rnew, *sn, *g, *Rrot, *y, *qpart, *sbuf, *V0;
  const double2** srcptr;
  double* scale;
  double* res_exp;
  double2* hcol;           // per slot: t Hessenberg columns of maxZ + 2 (when they exceed shared memory)
  // per slot, new column b, plane q: (Re w, Im w - Re w, Re w + Im w) of the new columns, the
  // operand of the inner products in Gauss's three-multiplication form (slots x t x 3 x D)
  double* Wp;
  // Gram-Schmidt on the tensor cores (gs_tc.cu, hh_opts.gs_tensor): every basis vector and
  // every new column cut into eight 7-bit slices held exactly in bf16, see gs_tc.cu
  int gst;                 // 1: the tensor-core Gram-Schmidt kernels run
  int Dp;                  // node count padded to a multiple of 768
  int NU;                  // rows of a vector's coefficient image: 20 t rounded up to 16
  unsigned char** VSptr;   // per slot, basis vector a: its slice images (64 Dp bytes)
  unsigned char** VScur;   // per slot: this iteration's block of slice images (t vectors)
  unsigned char* V0S;      // per slot: slice images of the first basis vector
  int* vexp;               // per slot, basis vector a: exponent e with max |v_a| < 2^e
  int *vnew0, *vnew1;      // per slot: basis vectors [vnew0, vnew1) still to be sliced
  unsigned long long* vmaxb;  // per slot, vector of the block: bits of max |entry|
  unsigned long long* wmaxb;  // per slot, new column: bits of max |entry|
  unsigned char* CB;       // per slot, basis vector a: coefficient image (NU x 32 bytes)
  int* cexp;               // per slot, new column: exponent of its coefficient images
};

}  // namespace hh
