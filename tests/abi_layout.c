/* Prints the size and field offsets of the C-ABI structs of include/hs.h, one "name size offsets..." line
 * per struct, for tests/test_abi.py to compare with the ctypes binding. */
#include <stddef.h>
#include <stdio.h>

#include "hs.h"

#define OFF(T, f) (long)offsetof(T, f)

int main(void) {
  printf("hs_z2_tensor %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld\n", (long)sizeof(hs_z2_tensor),
         OFF(hs_z2_tensor, D), OFF(hs_z2_tensor, n_even), OFF(hs_z2_tensor, n_odd), OFF(hs_z2_tensor, basis),
         OFF(hs_z2_tensor, dtype), OFF(hs_z2_tensor, data), OFF(hs_z2_tensor, capacity_bytes),
         OFF(hs_z2_tensor, v_even), OFF(hs_z2_tensor, v_odd), OFF(hs_z2_tensor, h_even), OFF(hs_z2_tensor, h_odd));
  printf("hs_env %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld\n", (long)sizeof(hs_env),
         OFF(hs_env, D), OFF(hs_env, chi_max), OFF(hs_env, chi_even), OFF(hs_env, chi_odd), OFF(hs_env, q_even),
         OFF(hs_env, q_odd), OFF(hs_env, basis), OFF(hs_env, precision), OFF(hs_env, gemm_backend),
         OFF(hs_env, moves), OFF(hs_env, log_norm_C), OFF(hs_env, log_norm_T), OFF(hs_env, C), OFF(hs_env, T),
         OFF(hs_env, C_bytes), OFF(hs_env, T_bytes), OFF(hs_env, eig_mode), OFF(hs_env, dtype));
  printf("hs_move_info %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld\n", (long)sizeof(hs_move_info),
         OFF(hs_move_info, chi_even), OFF(hs_move_info, chi_odd), OFF(hs_move_info, n_even), OFF(hs_move_info, n_odd),
         OFF(hs_move_info, lam_max), OFF(hs_move_info, lam_cut), OFF(hs_move_info, lam_next), OFF(hs_move_info, gap),
         OFF(hs_move_info, log_norm_C), OFF(hs_move_info, log_norm_T), OFF(hs_move_info, gemm_flops),
         OFF(hs_move_info, flags), OFF(hs_move_info, subspace_iters), OFF(hs_move_info, subspace_reason),
         OFF(hs_move_info, subspace_resid));
  printf("hs_hotrg_info %ld %ld %ld %ld %ld %ld %ld %ld\n", (long)sizeof(hs_hotrg_info), OFF(hs_hotrg_info, h_even),
         OFF(hs_hotrg_info, h_odd), OFF(hs_hotrg_info, side), OFF(hs_hotrg_info, discarded_left),
         OFF(hs_hotrg_info, discarded_right), OFF(hs_hotrg_info, log_norm), OFF(hs_hotrg_info, trace));
  printf("hs_env4 %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld\n", (long)sizeof(hs_env4),
         OFF(hs_env4, D), OFF(hs_env4, chi_max), OFF(hs_env4, chi_even), OFF(hs_env4, chi_odd), OFF(hs_env4, q_even),
         OFF(hs_env4, q_odd), OFF(hs_env4, basis), OFF(hs_env4, moves), OFF(hs_env4, C), OFF(hs_env4, T),
         OFF(hs_env4, C_bytes), OFF(hs_env4, T_bytes), OFF(hs_env4, log_norm_C), OFF(hs_env4, log_norm_T),
         OFF(hs_env4, svd));
  printf("hs_move4_info %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld %ld\n", (long)sizeof(hs_move4_info),
         OFF(hs_move4_info, direction), OFF(hs_move4_info, chi_even), OFF(hs_move4_info, chi_odd),
         OFF(hs_move4_info, m_even), OFF(hs_move4_info, m_odd), OFF(hs_move4_info, n_even), OFF(hs_move4_info, n_odd),
         OFF(hs_move4_info, s_max), OFF(hs_move4_info, s_cut), OFF(hs_move4_info, s_next), OFF(hs_move4_info, gap),
         OFF(hs_move4_info, gemm_flops));
  return 0;
}
