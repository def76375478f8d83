/*
 * md_flops.h -- algorithmic FP32 operation counts per unordered interacting
 * molecule pair, frozen from the expression trees of the site-site kernels
 * in paper_1408_4599_gb300/csrc/md_force.cu (mol_pair + elec_site).
 *
 * Counting rule: FMA = 2; add, sub, mul, compare/select = 1; rcp/rsqrt = 1
 * (the MUFU count is listed separately).  "Per unordered pair" means the
 * work that yields the pair energy, the pair virial, the force on both
 * molecules (equal and opposite) and the torque on both molecules, done
 * once -- i.e. the half-shell (Newton-3) kernel's count.  The full-shell
 * kernel executes the i-side part twice per pair; that repetition is not
 * counted as useful work.  The centre-of-mass distance test of an examined
 * candidate (12 FLOP) is overhead and is not counted either (§3: only ~16%
 * of the examined pairs interact).
 *
 * Building blocks (source expression trees):
 *   site vector x = X + d_a - d_b ............................ 6
 *   r^2 ...................................................... 5
 *   LJ: rcp 1, s2 1, s6 2, F/r 5, energy 5, force 3 ........... 17  (1 MUFU)
 *   accumulate the force on site a and on site b ............. 6
 *     => one LJ-LJ site pair ................................. 34
 *   QQ site pair: x 6, r^2 5, rsqrt 1, ir^2 1, xh 3,
 *     pa/pb/cab 15, u^2 u^3 2, law 44, U 1, radial coeff. 5,
 *     ua ub 2, force 18, e_a x e_b 9, torque on i 21,
 *     accumulate 6 ........................................... 139 (1 MUFU)
 *     + torque on j 21 ....................................... 160
 *   per molecule pair: total force 3 per site of j, energy 1,
 *     virial 6, virial diagonal 6; lever-arm torque of j
 *     9 per site of j.
 */
#ifndef MD_FLOPS_H
#define MD_FLOPS_H

/* single LJ site at the centre of mass (LJ / LJTS fluids):
 * r^2 5 + LJ 17 + accumulate 3 + energy 1 + virial 6 + diagonal 6 = 38 */
#define MD_FLOPS_PAIR_LJ1 38
#define MD_MUFU_PAIR_LJ1 1

/* 2CLJQ: 2 LJ sites + 1 linear quadrupole at the centre of mass:
 * 4 x 34 + 160 + 3 x 3 + 13 + 3 x 9 = 345 */
#define MD_FLOPS_PAIR_2CLJQ 345
#define MD_MUFU_PAIR_2CLJQ 5

/* distance test of one examined candidate (overhead, not counted above) */
#define MD_FLOPS_EXAMINED 12

#endif
