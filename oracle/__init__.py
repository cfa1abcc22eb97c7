"""Plain FP64 CPU oracle of the ddLPB energy and analytical forces.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package entry
file and the CPU-baseline leg of the benchmark may import anything from this
package; the product (the CUDA library and its Python binding) never does, and
shares no code, table or helper with it.

Every function follows a passage of Jha, Nottoli, Mikhalev, Quan and Stamm,
"Linear scaling computation of forces for the domain-decomposition linear
Poisson-Boltzmann method" (arXiv:2203.00552), cited by section and equation.

Modules: sph (Lebedev rules, real Y_lm, modified spherical Bessel functions),
ddlpb (the discrete problem, its solves, energy and forces), fmm (the tree
approximation of the Yukawa far field used by the FMM mode, fmm_order > 0, of
ddlpb: energy and solves only; parity of the GPU path is against the direct mode).
"""
