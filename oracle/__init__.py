"""FP64 CPU oracle for the LLG hot path of Zhu, "Grace: a cross-platform micromagnetic
simulator on graphics processing units" (arXiv:1411.2565).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code, header,
table or constant generator with the CUDA library: every quantity here is written
out plainly from the paper's equations (Sec. 2, Eqs. 1-3; Sec. 3 for the FFT
demag with zero padding, the six-neighbour exchange and the explicit Euler step)
and the readings of it stated in each function's docstring.

Modules:

* ``newell``   cell-averaged demagnetisation tensor (Newell-Williams-Dunlop form,
               Sec. 3 ref. [3]) with a far-field asymptote; pinned against the
               Aharoni prism factor, numerical quadrature and the point dipole.
* ``demag``    the demag field as a direct O(N^2) sum and as a zero-padded FFT
               convolution (Sec. 1 and Sec. 3).
* ``llg``      exchange, anisotropy, Zeeman, H_eff (Eqs. 1-2), the LLG right-hand
               side (Eq. 3), explicit Euler with |m| renormalised, energies (Eq. 1).
* ``adjoint``  the exact discrete adjoint of the FP64 Euler map, for gradients of a
               final-time loss with respect to per-cell applied field and Ms.

Arrays use the layout ``[3][nz][ny][nx]`` (x fastest), SI units, H in A/m.
"""
