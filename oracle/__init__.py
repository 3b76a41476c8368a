"""FP64 CPU oracle for the AIFMM factorisation and solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import or run anything in
this package.  The product (the CUDA library and its Python binding) never
calls it, and it shares no code with the CUDA path: it reads only the seeded
inputs of the top-level ``workloads`` module.

It is a plain, slow, sequential restatement of the method of Gujjula &
Ambikasaran, "Algebraic Inverse Fast Multipole Method" (arXiv 2301.12704):

* ``tree``      -- Sec. 2.1 (uniform 2^d tree) and Sec. 2.2 (admissibility,
                   neighbours N(i), interaction list IL(i)); distance-2 colours.
* ``kernels``   -- the interaction matrix A (Sec. 4 kernels).
* ``nnca``      -- Sec. 2.3 (eq. NCA, the operator list and Table 2) with an
                   ACA pivot search (the paper defers the search to its NNCA
                   reference; see the header of ``nnca``).
* ``extended``  -- Sec. 3.1 (unknowns x, y, z; equations X, Y; the extended
                   sparse matrix), as a dictionary of dense blocks.
* ``factor``    -- Sec. 3.2-3.5 (elimination, fill-ins, compress and redirect
                   with rank-revealing QR, Algorithm 2) and Sec. 3.6
                   (Algorithm 3, back substitution).
* ``h2``        -- the NNCA H^2 matrix-vector product and its dense form.

Parity status per function is stated in each module header.
"""
