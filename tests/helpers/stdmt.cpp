// Prints outputs of the C++ standard library's mersenne_twister_engine
// instantiations (std::mt19937, std::mt19937_64): a library routine used to pin
// the oracle.  Usage: stdmt <32|64> <seed> <discard> <count>
#include <cstdio>
#include <cstdlib>
#include <random>

int main(int argc, char** argv) {
    if (argc != 5) return 2;
    int bits = std::atoi(argv[1]);
    unsigned long long seed = std::strtoull(argv[2], nullptr, 10);
    unsigned long long skip = std::strtoull(argv[3], nullptr, 10);
    long count = std::atol(argv[4]);
    if (bits == 32) {
        std::mt19937 g(static_cast<std::mt19937::result_type>(seed));
        g.discard(skip);
        for (long i = 0; i < count; i++) std::printf("%u\n", static_cast<unsigned>(g()));
    } else {
        std::mt19937_64 g(seed);
        g.discard(skip);
        for (long i = 0; i < count; i++) std::printf("%llu\n", static_cast<unsigned long long>(g()));
    }
    return 0;
}
