"""NSSG (Navigating Satellite System Graph, arXiv 1907.06146) index construction and
search on one GB300 (sm_103a).

The compute path is the C-ABI library ``libssg.so`` (hand-written CUDA, declared in
``include/ssg.h``); :mod:`paper_1907_06146_gb300.ssg` is its thin Python binding and
:mod:`paper_1907_06146_gb300.synth` draws the seeded synthetic inputs.  Importing the
package loads nothing; the binding loads the library on first use and raises if it is
missing.
"""
__all__ = ["ssg", "synth"]
