"""CPU oracle for the LRDMC hot path — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the walker propagation and branching
step compute, written from the paper (Nakano, Sorella, Casula, "Load-Balanced
Diffusion Monte Carlo Method with Lattice Regularization", arXiv 2508.12033)
and from the plain definitions of the trial-wavefunction quantities:

* ``philox``       counter-based random numbers (Philox4x32-10, Salmon et al. 2011)
* ``wavefunction`` Slater-Jastrow values, ratios by freshly computed determinants
* ``hamiltonian``  lattice-regularised fixed-node Hamiltonian: hops, V_sf, W, e_L
* ``lrdmc``        load-balanced and conventional steps, reconfiguration, run loop
* ``estimator``    global population factor, weighted energy, blocked error bar,
                   a -> 0 extrapolation
* ``adjoint``      e_L and log|Psi_G| restated with PyTorch CPU tensors and
                   differentiated by autograd (nuclear coordinates, Jastrow)

It shares no code with the CUDA library and never imports it.  Only the test
suite, the smoke check and the benchmark's CPU-baseline leg may import it; the
product path must never route through it.

Parity status: every function is pinned by a test against something other than
itself (closed forms, brute force, invariants, exact diagonalisation, an
independent Philox implementation), except two readings of the paper that
only the agreement of the two implementations fixes ("parity unpinned"): the
E_0 update rule / estimator parameters, and which electrons the nodal cap
covers when several electrons are present (per electron or per
configuration).  The node-crossing pieces
themselves (removed hops, V_sf, the cap on an electron with such a hop) are
pinned for one electron, where both rules coincide, by exact
diagonalisation of the fixed-node lattice Hamiltonian of a nodal guiding
function.
"""
