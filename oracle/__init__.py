"""Plain FP64 CPU oracle for the truncated Wigner approximation (TWA) ensemble.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or calls it, and it imports
nothing from the CUDA library: the two share only the seeded input generators
of ``twa_inputs``.

Modules (each function cites the passage of arXiv:2310.07119 it follows):
  philox  - Philox4x32-10 counter-based generator (Salmon et al., SC'11) and
            the Box-Muller transform, used to draw the Wigner noise of Eq. sample.
  sp      - the normalized Schroedinger-Poisson system (Eq. mft_normed) and its
            pseudo-spectral split-step integrator (Sec. III.B.2), plus the
            conserved mass and energy used as pins.
  twa     - sampling of the stream ensemble (Sec. III.B.1, Eq. sample), the run
            loop, and the ensemble moments (Eq. Q, Eq. E[op], Sec. III.C).
  fock    - brute-force Fock-space evolution of the lattice Hamiltonian
            (Eq. eqn_Ham) for 2-4 modes, the exact quantum reference.
  kerr    - the single-mode quartic (Kerr) oscillator of Fig. 2 in closed form.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except ``twa.stable_growth_exponent`` (parity
partially pinned: the paper's kappa tensor, Eq. DefinitionKappa, is garbled, so
only the quadratic exponent of the early growth of Q is checked).
"""
