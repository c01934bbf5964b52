"""CPU FP64 oracle for tree field integration — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import or run anything in this package. The product
(``paper_2609_34025_b300``) never imports it, and it never imports the product:
the two share no code. Inputs come from the ``workloads`` generators only.

Contents
--------
``kernels``       f(x) of a kernel spec, evaluated in FP64 at the grid samples
                  f(k*delta) (Appendix "Distance quantization": the kernel is
                  sampled on the integer distance lattice).
``brute``         the plain definition (Eq. "integration" / Eq. "stad-target"):
                  out[u] = sum_v f(delta * dhat(u,v)) F[v], with dhat the sum of
                  quantised edge lengths q_e = max(1, round(w_e/delta)) on the
                  tree path; one traversal per target, FP64 accumulation.
                  Also the distance-binned correlation used for the gradient
                  with respect to kernel parameters.
``kernels``       also d f(k delta) / d theta for every analytic kind (pinned by
                  central differences of ``brute``).
``stad_literal``  the paper's StAd-TFI: the decomposition (DecomposeOffPathComponents,
                  ChooseBackbone), the table evaluators (ComputeGTerm / ComputeGTerm2DFFT,
                  the Hankel product), the cross term from Lemma "Cross-component
                  correction", the recursion of Eq. "stad-split" and the exponential
                  sweeps (CrossSubRoutineExp),
                  in FP64 with numpy FFTs, on grid units; it also reports the
                  decomposition arrays (projections, depths, anchors, backbone
                  coordinates) for bit-exact comparison with the planner.

Pins (tests/test_oracle_pins.py): f == 1 gives column sums; a unit path is a
Toeplitz matvec; star and uniform-path exponential closed forms; operator
symmetry; agreement with scipy's all-pairs shortest paths; the literal StAd
equals brute force on every labelled tree with up to 7 vertices; the
caterpillar closed form and the direct quadruple loop for G; the paper's logged
decompositions. Parity unpinned: none of the arithmetic; only the tie-break
choices of the decomposition (which diameter / centroid among equals) are fixed
by reading, not by the paper.
"""
