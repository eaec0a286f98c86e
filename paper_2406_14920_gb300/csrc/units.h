// Compilation units of the J/K class kernels: ERI_JK_UNIT(X, P, YLO, YHI) is
// bra pair class X (0..9 = ss ps pp ds dp dd fs fp fd ff), precision P
// (0 FP64, 1 FP32) and the ket classes YLO..YHI.  k_unit.cu is compiled once
// per entry (build.py reads this list), so the heavy register kernels of one
// bra class compile in parallel; plan.cu dispatches through the same list.
#define ERI_JK_UNITS(U) \
  U(0, 0, 0, 0)         \
  U(0, 1, 0, 0)         \
  U(1, 0, 0, 1)         \
  U(1, 1, 0, 1)         \
  U(2, 0, 0, 2)         \
  U(2, 1, 0, 2)         \
  U(3, 0, 0, 3)         \
  U(3, 1, 0, 3)         \
  U(4, 0, 0, 4)         \
  U(4, 1, 0, 2)         \
  U(4, 1, 3, 4)         \
  U(5, 0, 0, 5)         \
  U(5, 1, 0, 2)         \
  U(5, 1, 3, 5)         \
  U(6, 0, 0, 6)         \
  U(6, 1, 0, 3)         \
  U(6, 1, 4, 6)         \
  U(7, 0, 0, 7)         \
  U(7, 1, 0, 1)         \
  U(7, 1, 2, 3)         \
  U(7, 1, 4, 5)         \
  U(7, 1, 6, 7)         \
  U(8, 0, 0, 8)         \
  U(8, 1, 0, 3)         \
  U(8, 1, 4, 8)         \
  U(9, 0, 0, 9)         \
  U(9, 1, 0, 9)

// Compilation units of the gradient kernels: ERI_GRAD_UNIT(X, P) is bra pair
// class X with every ket class, precision P (g_unit.cu, compiled per entry).
#define ERI_GRAD_UNITS(U) \
  U(0, 0) U(0, 1) U(1, 0) U(1, 1) U(2, 0) U(2, 1) U(3, 0) U(3, 1) U(4, 0) U(4, 1) \
  U(5, 0) U(5, 1) U(6, 0) U(6, 1) U(7, 0) U(7, 1) U(8, 0) U(8, 1) U(9, 0) U(9, 1)
