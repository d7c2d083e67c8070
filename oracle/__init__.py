"""FP64 CPU oracle of the multiscale S-fraction reduced-order method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the native library and its
Python binding) may import, call, link or run anything in this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` use it.

It restates the paper (Druskin, Mamonov, Zaslavsky, "Multi-scale S-fraction
reduced-order models for massive wavefield simulations") step by step in plain
NumPy/SciPy, FP64, in the paper's order and notation, and shares no code with
the CUDA path.  Only the seeded input generators (``synth``) serve both.

Modules
-------
``fine``       fine-grid assembly (Section 1) and the fine leapfrog.
``partition``  coarse cells, operator splitting (Section 2, Eq. splitN_c),
               corner-set removal (Section 3, Appendix B), I/O faces.
``rom``        face bases (Section 4.1; DCT reading and the frequency-limited
               Gramian of Eq. trgr), rational Krylov ROM (Section 4.2,
               Eq. npks/tfprj), block Lanczos (Appendix C, Eq. NtDtri),
               S-fraction coefficients (Eq. GammaTrans), face masses
               (Remark Sinsubspace, Eq. bdrytstep), projected sources/receivers,
               the per-cell layer-count rule of the dipping-layer workload.
``online``     on-line leapfrog of the coupled ROM (Algorithm alg1red stage 2,
               Eqs. intrtstep_td, bdrytstep, solatrec) and its discrete energy.
``freq``       frequency-domain coupled ROM (Algorithm alg2red) and transfer
               functions of cells and skeleton.
``elastic``    VTI elastic fine-grid pencil (Q1 elements, lumped mass, Thomsen's
               parameters), the first step of the elastic workload (Section 7).
``c_leapfrog`` the ROM and fine-grid leapfrog loops again in plain C with OpenMP
               (``c/leapfrog.c``), checked against ``online`` / ``fine``; the
               host-core timing path of the bench's CPU baseline.

Pins: ``tests/test_oracle_*.py`` check every function against closed forms the
paper prints, invariants it states, and brute force on tiny inputs.
"""
