"""FP64 CPU oracle for the DELIMIT spherical layers (Koppers & Merhof, arXiv:1808.01517).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / ``--impl reference`` leg use it.  It shares no code, tables or
constants with the CUDA library; both sides are fed the same seeded inputs from
``paper_1808_01517_gb300.synth``, which contains none of the method's
arithmetic.

Modules
-------
sh      real even-order SH basis, Laplace-Beltrami regularised pseudo-inverse,
        Signal2SH / SH2Signal and their adjoints (Sec. 2.2).
lsc     local spherical convolution: kernel geometry, neighbour and window
        tables, the literal resample -> point-wise product -> SH projection
        forward, the algebraically collapsed forward, and analytic gradients
        (Sec. 2.3 and "Extension to multiple b-values").

Every function is plain numpy in float64 and follows the paper's order of
steps; library primitives (matmul, einsum, Cholesky, QR) serve as single steps.
Where the paper is silent or garbled, the reading taken is stated in the
function's docstring.
"""
