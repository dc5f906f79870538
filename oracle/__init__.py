"""FP64 CPU oracle for the PAW finite-element Chebyshev filter.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the paper's equations that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` may import it.  The product path
(the C-ABI library and its Python binding) never calls it and shares no code
with it: not the quadrature tables, not the basis, not the mesh numbering.

Modules
-------
fe      Section 2.2 / 4.1: GLL/Gauss rules, Lagrange basis, periodic hex mesh,
        cell matrices (Eqs. FEM Ham entries, FEM S_loc entries, FEM Cmatrix),
        lumped GLL mass M_D, synthetic potential and projectors.
ops     Eqs. FE nonlocal contribution, Sinvapprox, Delta Sinv: H, S, exact
        S^-1 (Woodbury on the consistent mass), approximate S^-1.
cheb    Eqs. ChFSI recurrance / recurrance2, Eqs. RChFSI residual 0/1 and
        Algorithm 2 (residual-based Chebyshev filtered subspace).
rr      Algorithm 1 steps 4-6 (Rayleigh-Ritz), residual norms (Sec. 4),
        generalised Lanczos bounds, dense brute-force eigensolve.
grad    derivative of tr(X^T H X) with respect to V at quadrature points and
        to the PAW coupling matrices Delta_H.
kpoint  the same operators at a Bloch wavevector k (Eq. hij with the 1/2 |k|^2
        and -i k . grad terms, Bloch phases of Eqs. FE nonlocal contribution /
        FEM Cmatrix): complex H(k), S(k), exact and approximate S(k)^-1.

Parity status of each function is stated in its docstring ("pinned by ..."
naming the test in ``tests/test_oracle_*.py``); functions without a pin say
"parity unpinned".
"""
