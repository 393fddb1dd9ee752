"""Plain FP64 CPU oracle for the hp-DG subspace-correction solver.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library: it assembles the sparse DG matrix, the conforming prolongation, the
low-order-refined matrix and the block smoother explicitly from their
definitions, and runs PCG with them.

Modules
    basis      Gauss-Lobatto / Gauss-Legendre rules and Lagrange polynomials
    topology   faces, sub-faces, hanging vertices and master edges of a 2D mesh
               (the domain is the union of the leaves: holes allowed)
    topology3  sub-faces of a 3D mesh of cubes
    dg         SIPG and BR2 matrices, 2D and 3D (Section 2, Eq. fe-problem; Section 4.4)
    space      conforming prolongation P, V_J / V_e classification (Section 3)
    space3     the same built from master entities, any dimension (cube meshes)
    geometry   mapped and curved elements: a bilinear or caller's map of the
               lattice domain, physical gradients, weights and normals
    lor        low-order-refined matrices (Section 3.4), squares and cubes
    amg        the deterministic smoothed-aggregation V-cycle used for LOR
    solver     the additive preconditioner B and PCG (Section 4.1)
    rhs        load vectors: the synthetic sine right-hand side, a given f,
               and weakly imposed Dirichlet data (SIPG)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, manufactured solutions, invariants, hand-worked cases or brute
force.  The smoothed-aggregation AMG has no counterpart in the paper (the paper
uses BoomerAMG without stating its parameters), so it is pinned against its own
stated algorithm: hand-worked aggregations and prolongator entries
(tests/golden/amg_aggregation.txt), the error-propagation form of the V-cycle,
symmetry, exactness on a single level and the Galerkin identity.
dg.element_rows is pinned against the rows of dg.assemble, and
rhs.load_vector against closed-form integrals within the Gauss rule's error
bound.
"""
