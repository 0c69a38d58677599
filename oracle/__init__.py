"""Plain, slow, CPU-only FP64 oracle for the parallel-TEBD hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` use it.  It shares no code with
the CUDA library (``paper_2401_05301_gb300/``) and imports nothing from it.

Modules
-------
model   eq. (1) Hamiltonian, its three-site split, and exact gates
tebd    second-order TEBD on a Vidal Gamma-lambda MPS stored in B-form
ed      exact diagonalisation: dense Trotterised evolution and the fixed-N sector
free    U = 0 free bosons / hard-core free fermions: one-body propagators and
        the uniform-chain Bessel closed forms
supersite  the paper's super-site scheme (pairs of sites, d_eff = d^2, NN gates,
        one SVD per gate), the next variant after the three-site path
u1      the three-site update with U(1)-symmetric decompositions (charge-labelled
        bonds, block-by-block SVDs, rule T on the merged spectrum), as the paper runs it
randomized  truncation by a randomized range finder (the cheaper SVD of Sec. V),
        test matrices passed in

Every function cites the passage of the paper (arXiv:2401.05301) it follows.
Where the paper is silent, the reading taken is stated in the docstring.
"""
