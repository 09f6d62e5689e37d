"""ProbeSim CPU oracle -- test infrastructure only.

A plain, slow, single-threaded FP64 restatement of ProbeSim (Liu et al., PVLDB 11(1) 2017) used to
check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import it; the library never does.  It shares no code with the CUDA path.

Modules:
  ``core``          ctypes wrapper of ``probesim_oracle.c`` (Philox, walks, PROBE, Alg. 1, Alg. 4, top-k, pair MC)
  ``power_method``  all-pairs SimRank by the Power Method, Eq. 6
  ``enumerate``     exact expectations on tiny graphs: first-meeting probability (Def. 4, Lemma 2) by
                    enumerating walks, and the expectation of the estimator over all walks (Lemma 1)
  ``build``         compiles ``probesim_oracle.c`` with gcc

Parity pins (the ``-m "not gpu"`` tests under ``tests/test_oracle_*.py``): the worked PROBE example and
Table 2 of the paper on the toy graph in ``tests/golden/``, closed forms of Eq. 1, Lemma 1 and Lemma 2
by enumeration, Thm. 1 statistically against the Power Method, the pruning lemmas' one-sided bounds,
the randomized PROBE's mean (Lemma in the proof of Thm. 3), and Philox by statistics and avalanche.
"""
