"""FP64 CPU oracle for the VMC-PEPS hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference legs
of ``bench.py`` may import this package.  The product path (the CUDA library and its
Python binding) never imports it and shares no code with it.

Modules
-------
philox  Philox4x32-10 counter-based generator (published definition).
vmc     boundary-MPS contraction with variational truncation, three- and four-line
        environments, sequential Metropolis sweep, E_loc, G = Delta/Psi, gradient
        and sign-SGD (arXiv:1908.09359, Sec. II, Algorithm 1, App. B, App. C).
exact   brute-force amplitudes and S^z = 0 enumeration for small lattices.
proposal        the learned band proposal and its Metropolis-Hastings step.
random_nnasp    the random-NNASP scheme of Sec. II A (exact transition matrices and
                attempt-by-attempt replay).
spin_inversion  Phi(S) = Psi(S) + Psi(S-bar): |Phi|^2 sweep, E^Phi, G^Phi (Sec. II B).
simple_update   simple-update imaginary-time evolution with NN and NNN gates (App. A).

Every function is pinned by the CPU tests (tests/test_oracle_*.py) to something
other than itself: known-answer vectors, brute force, closed forms, invariants and
finite differences.  Parity of finite-Dc results at L >= 8 against the paper itself
is unpinned (the paper prints no such numbers); those results are pinned only through
the exactness of the same code at Dc >= D^(L/2) and through the invariants.
"""
