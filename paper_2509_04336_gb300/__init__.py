"""GB300-native batched acceptance-walk nested sampler for gravitational-wave inference.

Importing the package loads nothing native; ``paper_2509_04336_gb300.gwns`` is the binding
to the C-ABI library ``libgwns.so`` and fails loudly when it is missing.
"""
