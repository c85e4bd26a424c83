"""The oracle: test infrastructure, not product code.

A plain, slow, obviously correct CPU restatement of what the library
computes, written from the paper (Peise, Fabregat-Traver, Bientinesi, "On the
Performance Prediction of BLAS-based Tensor Contractions"):

* ``contraction``  the FP64 contraction of Section 1 (nested loops in C);
* ``algorithms``   the algorithm generator of Section 2 / Table 1;
* ``prediction``   the integer cache analysis of Section 3;
* ``chain``        three-operand chains (Section 3.2's multi-kernel trees),
                   by the direct sum over the whole index space.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call, link or execute anything in this folder.  It
shares no code with the CUDA library and imports nothing from it.
"""
