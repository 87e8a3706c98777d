"""CPU oracle for the convex-programming LDS / LTDS method (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` may import it.  It shares no code with the CUDA path and imports
nothing from the product package; the tests feed both sides the same seeded
inputs.

It is written plainly and slowly from the paper (arXiv 2504.10937, "Finding
Locally Densest Subgraphs: Convex Programming with Edge and Triangle Density"):

* :mod:`oracle.graph`      - G, G[S], E(S), T, core and tr-core numbers
                             (Sec. 3, Def. 6, Def. 11);
* :mod:`oracle.fw`         - Frank-Wolfe for CP(G) (Alg. 1, Eq. 2) and for the
                             triangle program (Alg. 6, Eq. 4), exactly (rational
                             and integer-scaled) and in binary64 / binary32;
* :mod:`oracle.extract_sg` - stable groups and compact-number bounds (Alg. 2,
                             Def. 5, Def. 12, Lemma 4, Lemma 8);
* :mod:`oracle.prune`      - the two pruning rules (Alg. 3, Cor. 1, Lemma 5);
* :mod:`oracle.flow`       - exact integer max-flow / maximal min-cut (Dinic);
* :mod:`oracle.verify`     - IsDensest, IsLDS, IsLTDS, ExtMaximal (Sec. 5.4,
                             Alg. 4, Alg. 7, Alg. 8);
* :mod:`oracle.ldscvx`     - the LDScvx / LTDScvx driver (Alg. 5, Sec. 6);
* :mod:`oracle.decomp`     - exact compact numbers through the density-friendly
                             decomposition (Thm. 1, Thm. 4; Lemmas 2-3, Thm. 3)
                             and the LDS / LTDS sets they determine;
* :mod:`oracle.brute`      - the definitions themselves by exhaustive
                             enumeration of vertex subsets (Defs. 1-4, 7-10).

Which parts are pinned by what is recorded in each module's header.
"""
