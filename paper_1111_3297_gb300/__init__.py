"""GB300-native odd-only segmented sieve of Eratosthenes (Jarai & Vatai 2011 parameterisation)."""
