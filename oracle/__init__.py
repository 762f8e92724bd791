"""CPU oracle of the FFT momentum power-spectrum estimator (Pan, arXiv:2005.06170).

TEST INFRASTRUCTURE. Plain, slow FP64 code written from the paper's equations,
used to check the GPU library. Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import it. The GPU library (the
``paper_2005_06170_gb300`` package and its CUDA sources) neither imports nor links
anything here, and nothing here calls the GPU library.

Modules:
    bspline    - B-spline and orthonormalised (Battle-Lemarie) kernel definitions
    deposit.c  - FP64 B-spline assignment of particles to the grid (plain C)
    estimator  - moments, assignment, FFT, shot noise, deconvolution, binning,
                 bulk-flow variant (Secs. 2 and 3 of the paper)
    direct     - the BL function deposited in real space (whole, or truncated to a
                 radius: the oracle of the direct truncated deposit), and brute-force
                 references that pin the above (brute-force DFT, full-sphere binning)
    mu         - the spectra binned in (|k|, mu) about the bulk flow or a direction
                 (Sec. 2.2 and Sec. 3.2: the mu-dependent shot noise and the imaginary
                 cross spectrum that shell averages cancel)

Parity unpinned: nothing. Every function above is checked in tests/test_oracle_*.py
against closed forms, brute force or exact identities.
"""
