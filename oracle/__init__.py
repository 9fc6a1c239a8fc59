"""CPU oracle for the macromodel + AIM matrix-vector product (test infrastructure).

This package is test infrastructure: only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it.  The product (the C-ABI
library and its Python binding) never calls into it.

It is a plain, slow, complex128 restatement of the paper (Patel, Triverio,
Hum, "A Macromodeling Approach to Efficiently Compute Scattering from Large
Arrays of Complex Scatterers", arXiv 1712.02443):

* Sec. II   -- RWG / dual (Buffa-Christiansen) expansions, the Stratton-Chu
               matrices of eqs. (EFIEdiscretized1), (EFIEdiscretized2) and the
               macromodel T, A, B of eqs. (Hdiscretized1), (JM), (JABE), (Tm1);
* Sec. III  -- block-diagonal T, A, B for an array, reuse for identical elements;
* Sec. IV   -- exterior EFIE, D, G^(E^,J^), excitation, final system;
* Sec. V    -- AIM: projection, FFT convolution, interpolation, precorrected
               near field; GMRES.

Every function cites the passage it follows.  It shares no code with the CUDA
library: only the seeded input generators (meshes, angles, random vectors) of
``paper_1712_02443_gb300.workloads`` serve both.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, brute-force quadrature, Mie series, moment exactness, brute
force convolution, precorrection exactness).  The absolute accuracy of the
macromodel against a full MoM solve is pinned only to discretisation level,
which is the paper's own claim (exact up to discretisation, Sec. II).
"""
