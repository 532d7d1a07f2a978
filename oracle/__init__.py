"""Oracle: a plain, slow, FP64 CPU restatement of the simplex-grid hash encoding.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
Python binding, the serving loop) imports, calls or links anything in this
package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code, constant table or helper with
the CUDA path; both sides only share the seeded input generators, which hold
none of the method's arithmetic.

Every function cites the passage of the paper (Wen & Yang, "Efficient Encoding
of Graphics Primitives with Simplex-based Structures", arXiv 2311.15439) that it
restates.  Where the paper is silent the reading taken is stated at the
function.  Modules:

* ``lattice``  -- skew / unskew (Eq. 2, Eq. 3), level resolutions and the
  scale adjustment (Sec. 5.1), simplicial subdivision (Sec. 2.2 b, Sec. 4.2,
  Remark 2), barycentric weights (Sec. 4.3), the vertex hash (Sec. 5 a).
* ``encoding`` -- the multiresolution simplex encoding forward and backward
  (Sec. 5 a-e) and the 2^d multilinear grid comparator (Algorithm 1).
* ``mlp``      -- the tiny fully connected ReLU network, its backward pass and
  the L2 loss (Sec. 5 d-e, Sec. 6.1).
* ``adam``     -- the Adam update used to train tables and weights.
* ``render``   -- volumetric rendering with the encodings: ray samples, the
  quadrature of Eq. 5, spherical harmonics of the view direction (Sec. 6.2).
* ``geometry`` -- brute-force and closed-form facts used only to pin the
  oracle itself (Theorems 1-5, Lemma 4, Sec. 5.2 volume ratio).

Parity status per function is listed in each module docstring; the hash and
the Adam skip rule follow the Instant-NGP backbone the paper adopts (Sec. 5)
because the paper itself does not define them.
"""
