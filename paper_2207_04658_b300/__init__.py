"""paper_2207_04658_b300 -- quantized MLS-MPM on B300 (sm_103a).

The CUDA library (``libqmpm.so``) is loaded on first use by :mod:`.qmpm`; importing the
package itself loads nothing, so the seeded scene generators in :mod:`.scenes` can be
used without a GPU.
"""
