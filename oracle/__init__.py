"""FP64 single-threaded CPU oracle of the Cahn-Hilliard ensemble time-stepper.

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's CPU-baseline
leg.  The product library never imports it.
"""
