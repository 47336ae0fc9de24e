"""The oracle: a plain, slow FP64 CPU implementation of the axion Monte-Carlo
hot path, written from the paper (emission, absorption, detailed balance,
variance control, feedback and temperature evolution).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` may import or run anything
under ``oracle/``. The product path (the CUDA library and its Python binding)
never does, and the oracle never imports the product package: the two share
no code.

Parity status per function (details in each module's header):
* philox        - pinned (published known-answer vectors)
* spectra       - pinned (closed-form means, KS tests, Table II bremsstrahlung peaks)
* plasma        - pinned except the absolute bremsstrahlung emissivity, which
                  is parity unpinned (Table II's bremsstrahlung Q^R is not
                  reproducible from the printed fit)
* poisson       - pinned (scipy Poisson CDF, pmf chi-square)
* step          - pinned (conservation identities, steady states, unbiasedness)
* tally         - pinned (normalisation, closed forms)
* surrogate     - pinned (quantiles and emissivity integrals by scipy
                  quadrature, Primakoff limits, Debye map, MLP gradients by
                  finite differences, Adam's first step)
"""
from . import constants, philox, spectra, plasma, poisson, step, surrogate, tally  # noqa: F401
