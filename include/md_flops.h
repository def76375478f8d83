/*
 * md_flops.h -- algorithmic FP32 operation counts per unordered interacting
 * molecule pair, taken from the expression trees of the site-site code in
 * paper_1408_4599_gb300/csrc/md_pair.cuh (mol_pair, elec_site, law) and the
 * per-pair accumulation of csrc/md_forceop.cuh (ForceOp::pair).
 *
 * Counting rule: FMA = 2; add, sub, mul = 1; rcp / rsqrt = 1 (the MUFU
 * count is listed separately); a negation folded into an operand and a
 * product reused by common-subexpression elimination are not counted again.
 * "Per unordered pair" means the work that yields the pair energy, the pair
 * virial, the force on both molecules (equal and opposite) and the torque
 * on both molecules, done once -- the half-shell (Newton-3) kernel's count.
 * The full-shell kernel repeats the i-side part for the reversed pair; that
 * repetition is not counted as useful work.  The centre-of-mass distance
 * test of an examined candidate (MD_FLOPS_EXAMINED) is overhead and is not
 * counted either (§3: only ~16% of the examined pairs interact).
 *
 * The space-frame geometry of a molecule (site offsets R(q) d_a, axes
 * R(q) e_a) is a per-molecule quantity of the method; a kernel that forms
 * it again per pair (the linear-molecule path forms z_a u from the packed
 * axis u) does so as overhead, not counted.
 *
 * Building blocks (2CLJQ is compiled as a linear molecule with its
 * quadrupole at the centre of mass: site offsets are z_a u):
 *   lever arm X + z_a u, LJ sites of i ............................. 6
 *   LJ-LJ site pair: x = (X + z_a u_i) - z_b u_j 3, r^2 5, rcp 1,
 *     s^2 1, s^6 2, F/r 5, energy 5, site force 3, sum into a 3 .... 28  (1 MUFU)
 *   quadrupole-quadrupole pair (both at the COM: x = X): r^2 5,
 *     rsqrt 1, unit vector 3, p_a p_b cos_ab 15, law 38, strength
 *     6, energy 1, radial coefficient 5, axial coefficients 2, force
 *     18, e_a x e_b 9, orientation torque on i 21, sum into a 3 .... 127 (1 MUFU)
 *   per molecule pair: total force 3 per site of i, lever-arm
 *     torque u x (sum_a z_a f_a) 24, torque on j from the angular-
 *     momentum balance tau_j = -tau_i - X x F 12, accumulation of F
 *     and tau on i 6, energy 1, virial (trace and diagonal) 9,
 *     Newton-3 reaction on j 6.
 */
#ifndef MD_FLOPS_H
#define MD_FLOPS_H

/* single LJ site at the centre of mass (LJ / LJTS fluids):
 * r^2 5 + rcp 1 + s^2 1 + s^6 2 + F/r 5 + energy 4 + force 3
 * + accumulate F on i 3 + energy 1 + virial 9 + reaction on j 3 = 37 */
#define MD_FLOPS_PAIR_LJ1 37
#define MD_MUFU_PAIR_LJ1 1

/* 2CLJQ: 2 LJ sites + 1 linear quadrupole at the centre of mass:
 * 6 + 4 x 28 + 127 + 3 x 3 + 24 + 12 + 6 + 1 + 9 + 6 = 312 */
#define MD_FLOPS_PAIR_2CLJQ 312
#define MD_MUFU_PAIR_2CLJQ 5

/* distance test of one examined candidate (overhead, not counted above) */
#define MD_FLOPS_EXAMINED 12

#endif
