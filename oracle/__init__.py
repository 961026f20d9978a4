"""CPU oracle for the history-aware adaptive ROM (test infrastructure only).

This package is a plain, slow, FP64 NumPy/SciPy restatement of what the paper's
online step computes. It exists to check the CUDA library, and nothing in the
product path may import it: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. It shares no code, tables or helpers
with the CUDA path; both sides take their inputs from ``synth``.

Modules
-------
fv       FOM operators f(q) and J_f (Burgers, Euler/Rusanov) and the
         backward-Euler Newton step (Sec. 2 Eq. fom_lmm; Eq. be_residual_rom_section;
         App. B).
riemann  exact solution of the Riemann problem (used only to pin the Euler FOM).
rom      preprocessing, POD, Galerkin and DEIM-Galerkin reduced steps, QDEIM,
         feature-guided oversampling, the iSVD update (Algorithm 2) and the
         adaptive ROM driver (Algorithm 1).
adjoint  gradient of a terminal misfit of the adaptive Burgers ROM with respect
         to the viscosity and the initial-condition amplitude, in forward mode
         and as a checkpointed reverse sweep (no paper counterpart; pinned by
         finite differences of ``rom``).

Parity status: every function here is pinned by a test in ``tests/`` against a
closed form, an invariant, a library routine or brute force, except the
long-horizon adaptive trajectories themselves, whose values have no closed form
("parity unpinned" for the trajectory values; they are pinned only through
their ingredients).
"""
