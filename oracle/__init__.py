"""Plain FP64 CPU oracle for FS-FEM-T4 (face-based smoothed FEM, 4-node tets).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import or run anything in this
package.  The CUDA library never calls it, and it never calls the CUDA
library: the two share no code, headers, tables or constants.  The only
shared module is inputs/, which generates seeded meshes and load sets and
holds none of the method's arithmetic.

Modules
  fsfem  geometry (Eq. 10, Eq. 11, face normals), face topology (Section 3.2,
         Algorithm 1), smoothed gradients by Eq. 7 with the Gauss-point shape
         values of Table 1, the smoothed stiffness of Eq. 9, COO assembly with
         the sizes of Eq. 12 and its CSR form, loads and essential boundary
         conditions (STEP 5), dense checks (brute-force K, FEM-T4 K).
  solve  Jacobi-preconditioned CG in FP64 and a dense Cholesky solve.
  mlp    the learned coarse correction: residual pooling, 3-layer GELU MLP
         forward and backward in FP64, prolongation, Adam.
  coarse the two-level preconditioner: trilinear patch-centre coarse space,
         Galerkin coarse matrix, D^-1 + Pi A_c^-1 Pi^T, two-level PCG.
  nsfem  NS-FEM-T4 (node-based smoothing domains, Sec. 2.1): the stiffness
         assembled node by node from its definition.
  esfem  ES-FEM-T4 (edge-based smoothing domains, Sec. 2.1): the stiffness
         assembled edge by edge from its definition.
  recover strain and stress recovery for output (Sec. 3.4): face strains
         Bbar_k u_k (Eq. 7), stresses D eps_k, V_k-weighted nodal means, von
         Mises stress.

Every function is plain and slow on purpose; it cites the passage it follows.
"""
