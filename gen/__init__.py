"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds no part of the method's arithmetic: only problem constants,
sizes, index layouts of the variables, and seeded random draws.
"""
