"""Plain, slow FP64 CPU oracle for relativistic CCSD linear response (arXiv 2307.14296).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py`` may import or run anything in this package.  The CUDA library never
calls it and shares no code with it; the only common dependency is the seeded input generator
``synth`` (random numbers and layouts, no coupled-cluster arithmetic).

Modules (each function cites the passage it follows):
  ints     -- integral classes by index block, from the six stored classes
  det      -- definition level: second quantization in the N-electron determinant space
              (e^{-T} H e^{T} projections, FCI, sum-over-states response)
  ccsd     -- ground-state CCSD energy/residual/solver (spin-orbital Stanton-Gauss form)
  hbar     -- the similarity-transformed Hamiltonian intermediates of the SI (F, W, G, tau)
  sigma    -- right and left EOM-EE sigma vectors (SI Eqs. sigma_sin-ee ... _double-ee-left)
  props    -- xi^X, eta^X, EOM eta^X and the CC Hessian product t^X F (SI, linear response)
  deriv    -- derivative definitions of A, xi, eta, F by exact finite-difference stencils
  response -- Lambda solve, damped response solve (dense and Davidson), response function,
              polarizability and its derived quantities (Secs. 2.3-2.4, SI Davidson scheme)

Vectors over excitations use unique elements: singles t[i,a]; doubles are full antisymmetric
tensors t[i,j,a,b] whose independent entries are i<j, a<b.  Dot products over the vector space
count each unique doubles element once (1/4 of the full-tensor sum).

Parity status: every function is pinned by tests (see tests/test_oracle_*.py): the factorized
CCSD residual against the determinant-space definition, sigma/xi/eta/F against derivative
stencils of it, and the whole response chain against exact sum-over-states for two electrons
and against finite-field energies.  Nothing here is "parity unpinned".
"""
